"""Assembly, condensation, SpMV and solvers of the oracle (test infrastructure, FP64).

* ``assemble``: global matrix A_full = sum_e P_e^T A^e P_e (element matrices by
  the full-quadrature step-4 loop, Sec. 2.4), then the condensed operator
  K = C^T A_full C on the free DoFs and the identity on constrained DoFs
  (C expands free values to constrained ones: hanging -> weighted masters,
  Dirichlet -> 0).  The matrix-free operator of Sec. 3.6 has exactly this
  action.
* ``sampled_rows``: rows of K for chosen DoFs from their cells' element rows,
  for meshes whose full matrix does not fit in host memory.
* ``pcg``: Jacobi-preconditioned CG, x0 = 0, stop when ||r||_2 <= tol ||b||_2.
* ``chebyshev``: the degree-m Chebyshev-Jacobi preconditioner on [lo, hi].
* ``lanczos_lambda_max``: largest eigenvalue of D^-1 K from the CG tridiagonal.
* ``defect_correction``: FP64 residual and update around an FP32 inner solve
  (the single-precision solver with double-precision correction of Sec. 6.1).
"""
import numpy as np
import scipy.sparse as sp

from . import _native as nat
from .rules import basis_tables, gauss_legendre, gauss_lobatto

COEF_CONSTANT = 0
COEF_TRIG = 1


def element_matrices(mesh, nq, coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0), rows=None, cells=None):
    """Element stiffness matrices of the weak form of Eq. (1), with the coefficient a(x), by the full-quadrature cell loop of the step-4 listing (Sec. 2.4)."""
    k = mesh.k
    n = k + 1
    nodes = gauss_lobatto(k)
    xq, wq = gauss_legendre(nq)
    cv = mesh.cell_vertices if cells is None else mesh.cell_vertices[cells]
    cv = nat.f64(cv)
    C = cv.shape[0]
    par = nat.f64(np.asarray(coef_par, dtype=np.float64))
    if rows is None:
        out = np.zeros((C, n ** 3, n ** 3))
        nat.lib().or_cell_matrices(C, k, nq, nat.dp(nodes), nat.dp(xq), nat.dp(wq), nat.dp(cv),
                                   coef_kind, nat.dp(par), 0, None, nat.dp(out))
    else:
        r = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.zeros((C, len(r), n ** 3))
        nat.lib().or_cell_matrices(C, k, nq, nat.dp(nodes), nat.dp(xq), nat.dp(wq), nat.dp(cv),
                                   coef_kind, nat.dp(par), len(r), nat.ip(r), nat.dp(out))
    return out


def element_mass(mesh, nq):
    """Element mass matrices by the same full-quadrature cell loop (Sec. 2.4)."""
    k = mesh.k
    n = k + 1
    nodes = gauss_lobatto(k)
    xq, wq = gauss_legendre(nq)
    cv = nat.f64(mesh.cell_vertices)
    out = np.zeros((mesh.n_cells, n ** 3, n ** 3))
    nat.lib().or_cell_mass(mesh.n_cells, k, nq, nat.dp(nodes), nat.dp(xq), nat.dp(wq), nat.dp(cv),
                           nat.dp(out))
    return out


def quadrature_points(mesh, nq):
    """Physical quadrature points (C, nq^3, 3) and JxW (C, nq^3).

    The trilinear (Q1) map of each cell (Sec. 3.4).
    """
    xq, wq = gauss_legendre(nq)
    cv = nat.f64(mesh.cell_vertices)
    X = np.zeros((mesh.n_cells, nq ** 3, 3))
    J = np.zeros((mesh.n_cells, nq ** 3))
    nat.lib().or_cell_qpoints(mesh.n_cells, nq, nat.dp(xq), nat.dp(wq), nat.dp(cv), nat.dp(X), nat.dp(J))
    return X, J


def global_from_elements(mesh, Ae):
    """A_full = sum_e P_e^T A^e P_e as CSR; duplicates summed in (cell, i, j) order.

    Global assembly of the element matrices (Sec. 2.4): the matrix that the matrix-free operator of Sec. 3.6 never forms.
    """
    C, nd, _ = Ae.shape
    rows = np.repeat(mesh.cell_dofs, nd, axis=1).ravel()
    cols = np.tile(mesh.cell_dofs, (1, nd)).ravel()
    return sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=(mesh.n_dofs, mesh.n_dofs)).tocsr()


def constraint_matrix(mesh):
    """C with x_full = C x: identity on free DoFs, masters/weights on hanging, 0 on Dirichlet.

    The hanging-node constraints of Sec. 3.1 (Fig. 2) and the Dirichlet constraints, as applied in Sec. 3.3.
    """
    N = mesh.n_dofs
    is_c = np.zeros(N, dtype=bool)
    is_c[mesh.constrained] = True
    free = np.nonzero(~is_c)[0]
    r = list(free)
    c = list(free)
    v = [1.0] * len(free)
    for t, dof in enumerate(mesh.constrained):
        for p in range(mesh.cptr[t], mesh.cptr[t + 1]):
            r.append(dof)
            c.append(mesh.cmaster[p])
            v.append(mesh.cweight[p])
    return sp.csr_matrix((v, (r, c)), shape=(N, N)), is_c


def condense(mesh, A_full):
    """K = C^T A_full C (free rows/cols) + identity on constrained DoFs.

    Condensation of the constraints (Sec. 3.3).
    """
    Cm, is_c = constraint_matrix(mesh)
    K = (Cm.T @ A_full @ Cm).tocsr()
    K = K + sp.diags(is_c.astype(np.float64))
    K.sum_duplicates()
    K.sort_indices()
    return K.tocsr()


def assemble(mesh, nq, coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0)):
    """The condensed operator K whose action the matrix-free vmult computes (Sec. 3.6), assembled by the step-4 loop (Sec. 2.4)."""
    return condense(mesh, global_from_elements(mesh, element_matrices(mesh, nq, coef_kind, coef_par)))


def spmv(K, x):
    """y = K x with the oracle's plain CSR row loop.

    The action K x that the matrix-free operator of Sec. 3.6 reproduces.
    """
    K = K.tocsr()
    rp = np.ascontiguousarray(K.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(K.indices, dtype=np.int64)
    va = nat.f64(K.data)
    x = nat.f64(x)
    y = np.zeros(K.shape[0])
    nat.lib().or_csr_spmv(K.shape[0], nat.lp(rp), nat.lp(ci), nat.dp(va), nat.dp(x), nat.dp(y))
    return y


class CSR:
    """Pre-converted CSR arrays for repeated oracle SpMVs.

    Used for the action K x that the matrix-free operator of Sec. 3.6 reproduces.
    """

    def __init__(self, K):
        K = K.tocsr()
        self.n = K.shape[0]
        self.rp = np.ascontiguousarray(K.indptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(K.indices, dtype=np.int64)
        self.va = nat.f64(K.data)

    def __call__(self, x, y=None):
        x = nat.f64(x)
        if y is None:
            y = np.zeros(self.n)
        nat.lib().or_csr_spmv(self.n, nat.lp(self.rp), nat.lp(self.ci), nat.dp(self.va), nat.dp(x), nat.dp(y))
        return y


def sampled_rows(mesh, nq, dofs, x, coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0)):
    """(K x)[dofs] for a mesh without hanging nodes, from the element rows of each DoF's cells.

    Constrained entries of x are replaced by 0 (Dirichlet) before the product;
    constrained rows return x itself (identity rows).
    Entries of the action of Sec. 3.6 built from the element rows of the step-4 loop (Sec. 2.4).
    """
    if len(mesh.cmaster):
        raise NotImplementedError("sampled rows support Dirichlet-only meshes")
    n3 = mesh.cell_dofs.shape[1]
    is_c = np.zeros(mesh.n_dofs, dtype=bool)
    is_c[mesh.constrained] = True
    xf = np.where(is_c, 0.0, x)
    dofs = np.asarray(dofs, dtype=np.int64)
    # cells and local positions of each DoF
    cd = mesh.cell_dofs
    where = {int(d): [] for d in dofs}
    hit = np.isin(cd, dofs)
    for c, i in zip(*np.nonzero(hit)):
        where[int(cd[c, i])].append((c, i))
    y = np.zeros(len(dofs))
    for t, d in enumerate(dofs):
        d = int(d)
        if is_c[d]:
            y[t] = x[d]
            continue
        s = 0.0
        for c, i in where[d]:
            row = element_matrices(mesh, nq, coef_kind, coef_par, rows=[i], cells=[c])[0, 0]
            s += float(row @ xf[cd[c]])
        y[t] = s
        assert n3 == row.shape[0]
    return y


def cell_rhs(mesh, nq, coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0), fq=None):
    """Element right-hand sides (C, n^3): manufactured forcing, or f given at quadrature points.

    The right-hand-side integrals of the step-4 cell loop (Sec. 2.4).
    """
    k = mesh.k
    n = k + 1
    nodes = gauss_lobatto(k)
    xq, wq = gauss_legendre(nq)
    cv = nat.f64(mesh.cell_vertices)
    par = nat.f64(np.asarray(coef_par, dtype=np.float64))
    out = np.zeros((mesh.n_cells, n ** 3))
    if fq is None:
        nat.lib().or_cell_rhs(mesh.n_cells, k, nq, nat.dp(nodes), nat.dp(xq), nat.dp(wq), nat.dp(cv),
                              coef_kind, nat.dp(par), 0, None, nat.dp(out))
    else:
        f = nat.f64(fq)
        nat.lib().or_cell_rhs(mesh.n_cells, k, nq, nat.dp(nodes), nat.dp(xq), nat.dp(wq), nat.dp(cv),
                              coef_kind, nat.dp(par), 2, nat.dp(f), nat.dp(out))
    return out


def rhs(mesh, nq, coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0), fq=None):
    """b = C^T b_full on free DoFs, 0 on constrained DoFs.

    Condensed with the constraints of Sec. 3.3.
    """
    be = cell_rhs(mesh, nq, coef_kind, coef_par, fq)
    bfull = np.zeros(mesh.n_dofs)
    np.add.at(bfull, mesh.cell_dofs.ravel(), be.ravel())
    Cm, is_c = constraint_matrix(mesh)
    b = Cm.T @ bfull
    b[is_c] = 0.0
    return b


def distribute(mesh, x):
    """Fill constrained entries: hanging -> weighted masters, Dirichlet -> 0.

    Distribution of constrained values after the solve (Sec. 3.3).
    """
    Cm, is_c = constraint_matrix(mesh)
    xf = np.where(is_c, 0.0, x)
    return Cm @ xf


def diagonal(K):
    """Diagonal of the condensed operator: the Jacobi preconditioner of the CG solves (Sec. 3.5, Sec. 6.1)."""
    return K.diagonal().copy()


def l2_error(mesh, x, nq_err=None, exact="sinxyz"):
    """||u_h - u||_L2 with a (k+3)-point Gauss rule; u = sin(pi x) sin(pi y) sin(pi z) ("sinxyz", zero on
    every face) or u = sin(pi x) ("sinx", zero on the x faces, zero normal derivative on the others).
    Error of the Poisson problem of Sec. 2.4 against a manufactured solution."""
    k = mesh.k
    nq_err = nq_err or k + 3
    nodes = gauss_lobatto(k)
    xq, wq = gauss_legendre(nq_err)
    uc = nat.f64(distribute(mesh, x)[mesh.cell_dofs])
    cv = nat.f64(mesh.cell_vertices)
    e2 = nat.lib().or_l2_error_sq(mesh.n_cells, k, nq_err, nat.dp(nodes), nat.dp(xq), nat.dp(wq),
                                  nat.dp(cv), nat.dp(uc), {"sinxyz": 0, "sinx": 1}[exact])
    return float(np.sqrt(e2))


NOT_CONVERGED = 1
BREAKDOWN = 2


class SolveResult:
    """Outcome of the CG solves of Sec. 6.1."""
    def __init__(self, x, iterations, rel_residual, status, history=None, alphas=None, betas=None):
        self.x = x
        self.iterations = iterations
        self.rel_residual = rel_residual
        self.status = status
        self.history = history or []
        self.alphas = alphas or []
        self.betas = betas or []


def pcg(A, b, precond, tol=1e-10, max_it=100000, dtype=np.float64, x0=None):
    """Preconditioned CG (x0 = 0): stop when ||r||_2 <= tol ||b||_2.

    A and precond are callables on vectors of `dtype`; scalars are kept in
    `dtype` as well (float32 for the inner single-precision solve).
    The conjugate-gradient solver of Sec. 6.1 with a Jacobi or Chebyshev-Jacobi preconditioner (Sec. 3.5).
    """
    b = b.astype(dtype)
    x = np.zeros_like(b) if x0 is None else x0.astype(dtype).copy()
    r = b - A(x) if x0 is not None else b.copy()
    bnorm = float(np.sqrt(np.dot(b.astype(np.float64), b.astype(np.float64))))
    if bnorm == 0.0:
        return SolveResult(x, 0, 0.0, 0)
    z = precond(r)
    p = z.copy()
    rz = dtype(np.dot(r, z))
    hist, alphas, betas = [], [], []
    for it in range(1, max_it + 1):
        q = A(p)
        pq = dtype(np.dot(p, q))
        if not np.isfinite(pq) or pq <= 0:
            return SolveResult(x, it, np.nan, BREAKDOWN, hist, alphas, betas)
        alpha = dtype(rz / pq)
        x = x + alpha * p
        r = r - alpha * q
        rnorm = float(np.sqrt(np.dot(r.astype(np.float64), r.astype(np.float64))))
        hist.append(rnorm / bnorm)
        alphas.append(float(alpha))
        if not np.isfinite(rnorm):
            return SolveResult(x, it, np.nan, BREAKDOWN, hist, alphas, betas)
        if rnorm <= tol * bnorm:
            return SolveResult(x, it, rnorm / bnorm, 0, hist, alphas, betas)
        z = precond(r)
        rz_new = dtype(np.dot(r, z))
        beta = dtype(rz_new / rz)
        betas.append(float(beta))
        rz = rz_new
        p = z + beta * p
    return SolveResult(x, max_it, hist[-1], NOT_CONVERGED, hist, alphas, betas)


def lanczos_tridiagonal(alphas, betas):
    """Lanczos tridiagonal of the preconditioned operator from CG's coefficients.

    T_ii = 1/alpha_i + beta_{i-1}/alpha_{i-1},  T_{i,i+1} = sqrt(beta_i)/alpha_i.
    The eigenvalue estimate behind the Chebyshev interval (Sec. 3.5).
    """
    m = len(alphas)
    T = np.zeros((m, m))
    for i in range(m):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < m:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    return T


def lanczos_lambda_max(A, dinv, start, steps=15):
    """Largest eigenvalue estimate of D^-1 A after `steps` Jacobi-PCG steps from `start`.

    The eigenvalue estimate behind the Chebyshev interval (Sec. 3.5).
    """
    res = pcg(A, start, lambda r: dinv * r, tol=0.0, max_it=steps)
    m = min(len(res.alphas), len(res.betas) + 1)
    T = lanczos_tridiagonal(res.alphas[:m], res.betas[:m - 1])
    return float(np.linalg.eigvalsh(T).max())


def chebyshev(A, dinv, r, degree, lo, hi, dtype=np.float64):
    """z = p(D^-1 A) D^-1 r with 1 - lambda p(lambda) = T_m(sigma(lambda)) / T_m(sigma(0)).

    sigma(lambda) = (hi + lo - 2 lambda) / (hi - lo).  Computed by `degree`
    steps of the Chebyshev iteration for D^-1 A z = D^-1 r from z = 0
    (three-term recurrence; degree - 1 operator products).
    The Chebyshev-Jacobi smoother of Sec. 3.5, used as a CG preconditioner (Sec. 6.1).
    """
    theta = dtype((hi + lo) / 2.0)
    delta = dtype((hi - lo) / 2.0)
    sigma = theta / delta
    rho = dtype(1.0) / sigma
    r = r.astype(dtype)
    dinv = dinv.astype(dtype)
    d = dinv * r / theta
    z = d.copy()
    for _ in range(1, degree):
        res = r - A(z)
        rho_new = dtype(1.0) / (dtype(2.0) * sigma - rho)
        d = rho_new * rho * d + dtype(2.0) * rho_new / delta * (dinv * res)
        z = z + d
        rho = rho_new
    return z


def defect_correction(A64, A32, dinv64, b, inner_precond, tol=1e-10, inner_tol=1e-4,
                      max_outer=100, max_inner=10000):
    """Outer FP64 residual/update around an FP32 inner PCG (Sec. 6.1).

    x = 0; repeat: r = b - A64 x (FP64); stop if ||r|| <= tol ||b||;
    solve A32 d = r / ||r|| to inner_tol in FP32; x += ||r|| d.
    The single-precision solver inside a double-precision correction of Sec. 6.1.
    """
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    inner_total = 0
    for outer in range(max_outer + 1):
        r = b - A64(x)
        rn = float(np.linalg.norm(r))
        if rn <= tol * bnorm:
            return SolveResult(x, outer, rn / bnorm, 0, history=[inner_total])
        res = pcg(A32, (r / rn).astype(np.float32), inner_precond, tol=inner_tol,
                  max_it=max_inner, dtype=np.float32)
        inner_total += res.iterations
        if res.status == BREAKDOWN:
            return SolveResult(x, outer, rn / bnorm, BREAKDOWN, history=[inner_total])
        x = x + rn * res.x.astype(np.float64)
    return SolveResult(x, max_outer, rn / bnorm, NOT_CONVERGED, history=[inner_total])
