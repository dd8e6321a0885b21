"""1D rules on [0, 1] used by the oracle (test infrastructure, FP64).

The paper fixes tensor-product Lagrange elements on the reference cell
[0,1]^d (Sec. 3.1, Sec. 3.4) and quadrature formulas (Sec. 3.4); the
workloads name Gauss-Lobatto nodes and (k+1)-point Gauss quadrature.
Everything here is the textbook definition:

* Gauss-Legendre: the n roots of the Legendre polynomial P_n, weights
  2 / ((1 - t^2) P_n'(t)^2) on [-1, 1], mapped affinely to [0, 1];
* Gauss-Lobatto: {-1, 1} and the k-1 roots of P_k', mapped to [0, 1];
* Lagrange basis by the product formula.

Roots are found by Newton's method from Chebyshev starting points, in the
platform's extended precision (numpy longdouble: 64- or 113-bit
significand), and rounded to FP64 once at the end, after the affine map to
[0, 1]: each node and point is then the FP64 number nearest to the root it
is defined as (an FP64 Newton iteration in [-1, 1] followed by the map lost
up to three bits near the ends of the interval).  The weights are evaluated
from the rounded points.
"""
import numpy as np


def legendre(n, t):
    """P_n(t) and P_{n-1}(t) by the three-term recurrence (Bonnet).

    Building block of the Gauss and Gauss-Lobatto rules of the tensor-product elements (Sec. 3.1, Sec. 3.4).
    """
    t = np.asarray(t)
    if t.dtype != np.longdouble:
        t = t.astype(np.float64)
    p_prev = np.ones_like(t)
    if n == 0:
        return p_prev, np.zeros_like(t)
    p = t.copy()
    for m in range(2, n + 1):
        p_prev, p = p, ((2 * m - 1) * t * p - (m - 1) * p_prev) / m
    return p, p_prev


def legendre_deriv(n, t):
    """P_n'(t) = n (t P_n - P_{n-1}) / (t^2 - 1), valid for |t| < 1.

    Building block of the Gauss and Gauss-Lobatto rules (Sec. 3.1, Sec. 3.4).
    """
    p, pm = legendre(n, t)
    return n * (t * p - pm) / (t * t - 1.0), p


def _mirror(t_low, n):
    """Full symmetric node set on [-1, 1] from its negative half (t = 0 exact in the middle), in the
    precision of t_low."""
    t = np.zeros(n, dtype=t_low.dtype)
    h = n // 2
    t[:h] = t_low[:h]
    t[n - h:] = -t_low[:h][::-1]
    return t


def _newton_tol():
    """Step size below which the extended-precision Newton iteration stops (a few units of its last place)."""
    return 8 * float(np.finfo(np.longdouble).eps)


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1]: (points ascending, weights).

    The roots are symmetric about 0; the negative half is computed and
    mirrored so that the rule is exactly symmetric (midpoint exactly 1/2).
    The quadrature of the cell integrals (Sec. 2.4, Sec. 3.6).
    """
    if n < 1:
        raise ValueError("n >= 1")
    h = n // 2
    t = -np.cos(np.pi * (np.arange(h) + 0.75) / (n + 0.5)).astype(np.longdouble)  # ascending guesses
    for _ in range(100):
        if h == 0:
            break
        dp, p = legendre_deriv(n, t)
        dt = p / dp
        t = t - dt
        if np.max(np.abs(dt)) < _newton_tol():
            break
    t = _mirror(t, n)
    x = (0.5 * (t + 1.0)).astype(np.float64)  # one rounding, after the map to [0, 1]
    tr = 2.0 * x - 1.0  # the rounded points in [-1, 1] (exact)
    dp, _ = legendre_deriv(n, tr)
    w = 2.0 / ((1.0 - tr * tr) * dp * dp)
    return x, 0.5 * w


def gauss_lobatto(k):
    """Degree-k Gauss-Lobatto nodes (k+1 points, ascending) on [0, 1].

    Interior nodes are the roots of P_k'; Newton uses P_k'' from the
    Legendre equation (1 - t^2) P'' = 2 t P' - k (k+1) P.
    The nodes of the Lagrange shape functions (Sec. 3.1).
    """
    if k < 1:
        raise ValueError("k >= 1")
    if k == 1:
        return np.array([0.0, 1.0])
    h = (k - 1) // 2  # interior roots in the negative half
    t = -np.cos(np.pi * np.arange(1, h + 1) / k).astype(np.longdouble)
    for _ in range(100):
        if h == 0:
            break
        dp, p = legendre_deriv(k, t)
        d2p = (2.0 * t * dp - k * (k + 1) * p) / (1.0 - t * t)
        dt = dp / d2p
        t = t - dt
        if np.max(np.abs(dt)) < _newton_tol():
            break
    interior = _mirror(t, k - 1)
    nodes = np.concatenate((np.array([-1.0], dtype=np.longdouble), interior, np.array([1.0], dtype=np.longdouble)))
    return (0.5 * (nodes + 1.0)).astype(np.float64)  # one rounding, after the map to [0, 1]


def lagrange(nodes, j, x):
    """l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m).

    The 1D factors of the tensor-product shape functions (Sec. 3.1).
    """
    x = np.asarray(x, dtype=np.float64)
    v = np.ones_like(x)
    for m, xm in enumerate(nodes):
        if m != j:
            v = v * (x - xm) / (nodes[j] - xm)
    return v


def lagrange_deriv(nodes, j, x):
    """l_j'(x) = sum_{m != j} 1/(x_j - x_m) prod_{l != j, m} (x - x_l)/(x_j - x_l).

    The 1D factors of the tensor-product shape functions (Sec. 3.1).
    """
    x = np.asarray(x, dtype=np.float64)
    total = np.zeros_like(x)
    for m, xm in enumerate(nodes):
        if m == j:
            continue
        term = np.full_like(x, 1.0 / (nodes[j] - xm))
        for l, xl in enumerate(nodes):
            if l != j and l != m:
                term = term * (x - xl) / (nodes[j] - xl)
        total = total + term
    return total


def basis_tables(k, nq):
    """Values and derivatives of the degree-k GLL Lagrange basis at the nq Gauss points.

    Returns (gll_nodes, gauss_points, gauss_weights, V, Dv) with V[q, j] =
    l_j(xi_q) and Dv[q, j] = l_j'(xi_q).
    The 1D shape values and derivatives at the Gauss points that the tensor-product structure of Sec. 3.1 factorises.
    """
    nodes = gauss_lobatto(k)
    xq, wq = gauss_legendre(nq)
    V = np.array([[lagrange(nodes, j, x) for j in range(k + 1)] for x in xq])
    Dv = np.array([[lagrange_deriv(nodes, j, x) for j in range(k + 1)] for x in xq])
    return nodes, xq, wq, V, Dv
