"""Pins of the oracle's element matrices, assembly and solvers.

Each test checks the oracle against something other than itself: closed
forms, exact rational arithmetic, separable (Kronecker) integrals built from
numpy's polynomial class, invariants fixed by the mathematics (constants in
the kernel, symmetry, domain volume), library solvers, and manufactured-
solution convergence rates with a forcing derived independently by sympy.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, mesh, rules
from paper_1910_13247_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_q1_element_matrix_closed_form():
    ref = np.loadtxt(os.path.join(GOLDEN, "q1_laplace_unit_cube.txt")) / 12.0
    m = mesh.structured_mesh(1, 1, 1, 1)
    for nq in (2, 3):
        A = fem.element_matrices(m, nq)[0]
        assert np.allclose(A, ref, atol=1e-15)


def _exact_1d(k, h):
    """1D stiffness and mass matrices on [0, h] from numpy polynomial integrals."""
    nodes = rules.gauss_lobatto(k)
    n = k + 1
    polys = []
    for j in range(n):
        p = np.polynomial.Polynomial.fromroots([nodes[m] for m in range(n) if m != j])
        polys.append(p / p(nodes[j]))
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            pk = (polys[i].deriv() * polys[j].deriv()).integ()
            pm = (polys[i] * polys[j]).integ()
            K[i, j] = (pk(1) - pk(0)) / h
            M[i, j] = (pm(1) - pm(0)) * h
    return K, M


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_cartesian_element_is_kronecker_sum(k):
    hx, hy, hz = 0.5, 0.25, 2.0
    verts = np.array([[a * hx, b * hy, c * hz] for c in (0, 1) for b in (0, 1) for a in (0, 1)])
    m = mesh.Mesh(verts[None], np.zeros((1, (k + 1) ** 3), np.int64), (k + 1) ** 3,
                  np.zeros(0, np.int64), np.zeros(1, np.int64), np.zeros(0, np.int64), np.zeros(0), k)
    A = fem.element_matrices(m, k + 1)[0]
    Kx, Mx = _exact_1d(k, hx)
    Ky, My = _exact_1d(k, hy)
    Kz, Mz = _exact_1d(k, hz)
    # local index i1 + n (i2 + n i3): the x factor is the fastest (last) Kronecker factor
    ref = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    assert np.allclose(A, ref, atol=1e-13 * np.abs(ref).max())
    Mref = np.kron(Mz, np.kron(My, Mx))
    m2 = fem.element_mass(m, k + 1)[0]
    assert np.allclose(m2, Mref, atol=1e-14 * np.abs(Mref).max())


def _frac_poly_mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _frac_lagrange(nodes, j):
    p = [Fraction(1)]
    for m, xm in enumerate(nodes):
        if m != j:
            p = _frac_poly_mul(p, [-xm / (nodes[j] - xm), 1 / (nodes[j] - xm)])
    return p


def _frac_deriv(p):
    return [i * p[i] for i in range(1, len(p))]


def _frac_int01(p):
    return sum(c / (i + 1) for i, c in enumerate(p))


def _frac_element(k, h):
    """Exact rational Laplace element matrix on an axis-aligned box of sizes h (Fractions)."""
    nodes = [Fraction(i, k) for i in range(k + 1)] if k <= 2 else None
    n = k + 1
    L = [_frac_lagrange(nodes, j) for j in range(n)]
    dL = [_frac_deriv(p) for p in L]
    M1 = [[_frac_int01(_frac_poly_mul(L[i], L[j])) for j in range(n)] for i in range(n)]
    K1 = [[_frac_int01(_frac_poly_mul(dL[i], dL[j])) for j in range(n)] for i in range(n)]
    nd = n ** 3
    A = [[Fraction(0)] * nd for _ in range(nd)]
    for a in range(nd):
        ia = (a % n, (a // n) % n, a // (n * n))
        for b in range(nd):
            ib = (b % n, (b // n) % n, b // (n * n))
            s = Fraction(0)
            for d in range(3):
                t = Fraction(1)
                for e in range(3):
                    if e == d:
                        t *= K1[ia[e]][ib[e]] / h[e]
                    else:
                        t *= M1[ia[e]][ib[e]] * h[e]
                s += t
            A[a][b] = s
    return A


@pytest.mark.parametrize("k", [1, 2])
def test_two_cell_mesh_matches_rational_brute_force(k):
    # 2 x 1 x 1 cells of size (1/2, 1, 1): assembled matrix before constraints
    m = mesh.structured_mesh(2, 1, 1, k)
    A = fem.global_from_elements(m, fem.element_matrices(m, k + 1)).toarray()
    Ae = _frac_element(k, (Fraction(1, 2), Fraction(1), Fraction(1)))
    N = m.n_dofs
    ref = [[Fraction(0)] * N for _ in range(N)]
    for c in range(2):
        dofs = m.cell_dofs[c]
        for a in range(len(dofs)):
            for b in range(len(dofs)):
                ref[dofs[a]][dofs[b]] += Ae[a][b]
    ref = np.array([[float(v) for v in row] for row in ref])
    assert np.allclose(A, ref, atol=1e-14)
    # the numbering is the lattice rule: DoF I + Mx (J + My L)
    n = k + 1
    Mx, My = 2 * k + 1, k + 1
    for c in range(2):
        for i3 in range(n):
            for i2 in range(n):
                for i1 in range(n):
                    assert m.cell_dofs[c, i1 + n * (i2 + n * i3)] == (k * c + i1) + Mx * (i2 + My * i3)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_constants_in_kernel_symmetry_and_volume(k):
    nx = 3
    m = mesh.structured_mesh(nx, nx, nx, k, synthetic.deformed_vertices(nx, nx, nx))
    Ae = fem.element_matrices(m, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    A = fem.global_from_elements(m, Ae)
    ones = np.ones(m.n_dofs)
    scale = np.abs(A).max()
    assert np.abs(A @ ones).max() < 1e-12 * scale
    assert abs(A - A.T).max() < 1e-14 * scale
    K = fem.condense(m, A)
    assert abs(K - K.T).max() < 1e-14 * scale
    # mass sums to the volume of the deformed cube (exactly 1: the map is the identity on the boundary)
    Me = fem.element_mass(m, k + 1)
    assert abs(Me.sum() - 1.0) < 1e-13
    # constrained rows of K are identity rows
    Kd = K.tocsr()
    for c in m.constrained[:50]:
        row = Kd.getrow(c)
        assert row.nnz == 1 and row[0, c] == 1.0


def test_quadrature_points_follow_trilinear_map():
    nx = 2
    v = synthetic.deformed_vertices(nx, nx, nx)
    m = mesh.structured_mesh(nx, nx, nx, 2, v)
    X, J = fem.quadrature_points(m, 3)
    xq, wq = rules.gauss_legendre(3)
    # independent evaluation for cell 5 at q = (2, 0, 1)
    c = 5
    V = m.cell_vertices[c]
    s, t, u = xq[2], xq[0], xq[1]
    p = np.zeros(3)
    for vtx in range(8):
        a, b, e = vtx & 1, (vtx >> 1) & 1, (vtx >> 2) & 1
        p += (s if a else 1 - s) * (t if b else 1 - t) * (u if e else 1 - u) * V[vtx]
    assert np.allclose(X[c, 2 + 3 * (0 + 3 * 1)], p, atol=1e-15)
    assert abs(J.sum() - 1.0) < 1e-13


def _sympy_forcing():
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    u = sympy.sin(sympy.pi * x) * sympy.sin(sympy.pi * y) * sympy.sin(sympy.pi * z)
    a = 1 + sympy.Rational(1, 2) * sympy.sin(2 * sympy.pi * x) * sympy.cos(2 * sympy.pi * y) * z
    f = -(sympy.diff(a * sympy.diff(u, x), x) + sympy.diff(a * sympy.diff(u, y), y)
          + sympy.diff(a * sympy.diff(u, z), z))
    return sympy.lambdify((x, y, z), f, "numpy")


def test_builtin_forcing_matches_sympy():
    f = _sympy_forcing()
    m = mesh.structured_mesh(2, 2, 2, 2, synthetic.deformed_vertices(2, 2, 2))
    X, _ = fem.quadrature_points(m, 3)
    fq = f(X[..., 0], X[..., 1], X[..., 2])
    b1 = fem.rhs(m, 3, fem.COEF_TRIG, (1.0, 0.5))
    b2 = fem.rhs(m, 3, fem.COEF_TRIG, (1.0, 0.5), fq=fq)
    assert np.allclose(b1, b2, atol=1e-13)


def _solve_error(m, k, coef, par, fq=None):
    K = fem.assemble(m, k + 1, coef, par)
    b = fem.rhs(m, k + 1, coef, par, fq)
    x = spla.spsolve(K.tocsc(), b)
    return fem.l2_error(m, x)


@pytest.mark.parametrize("k,deformed,variable", [(1, False, False), (2, False, False), (3, False, False),
                                                   (2, True, True), (3, True, True)])
def test_manufactured_convergence_rate(k, deformed, variable):
    errs = []
    sizes = (2, 4, 8) if k < 3 else (2, 4, 6)
    f = _sympy_forcing() if variable else None
    for nx in sizes:
        v = synthetic.deformed_vertices(nx, nx, nx) if deformed else None
        m = mesh.structured_mesh(nx, nx, nx, k, v)
        fq = None
        if variable:
            X, _ = fem.quadrature_points(m, k + 1)
            fq = f(X[..., 0], X[..., 1], X[..., 2])
        coef = fem.COEF_TRIG if variable else fem.COEF_CONSTANT
        errs.append(_solve_error(m, k, coef, (1.0, 0.5) if variable else (1.0, 0.0), fq))
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(sizes[i + 1] / sizes[i]) for i in range(len(errs) - 1)]
    assert rates[-1] > k + 1 - 0.35, (errs, rates)


def test_pcg_matches_direct_solve():
    m = mesh.structured_mesh(4, 4, 4, 2, synthetic.deformed_vertices(4, 4, 4))
    K = fem.assemble(m, 3, fem.COEF_TRIG, (1.0, 0.5))
    b = synthetic.uniform_vector(m.n_dofs, 1)
    b[m.constrained] = 0
    dinv = 1.0 / fem.diagonal(K)
    res = fem.pcg(lambda v: K @ v, b, lambda r: dinv * r, tol=1e-12)
    assert res.status == 0
    xd = spla.spsolve(K.tocsc(), b)
    assert np.linalg.norm(res.x - xd) < 1e-9 * np.linalg.norm(xd)
    assert np.linalg.norm(b - K @ res.x) <= 1e-12 * np.linalg.norm(b) * 1.0001


def test_csr_spmv_matches_scipy():
    m = mesh.structured_mesh(3, 3, 3, 3, synthetic.deformed_vertices(3, 3, 3))
    K = fem.assemble(m, 4, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(m.n_dofs, 2)
    assert np.allclose(fem.spmv(K, x), K @ x, rtol=0, atol=1e-13 * np.abs(K @ x).max())


def test_sampled_rows_match_full_product():
    nx, k = 3, 3
    m = mesh.structured_mesh(nx, nx, nx, k, synthetic.deformed_vertices(nx, nx, nx))
    K = fem.assemble(m, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(m.n_dofs, 3)
    y = K @ x
    dofs = np.random.default_rng(0).choice(m.n_dofs, 40, replace=False)
    ys = fem.sampled_rows(m, k + 1, dofs, x, fem.COEF_TRIG, (1.0, 0.5))
    assert np.allclose(ys, y[dofs], atol=1e-13 * np.abs(y).max())


@pytest.mark.parametrize("degree", [2, 5, 6])
def test_chebyshev_closed_form_on_diagonal_operator(degree):
    lam = np.linspace(0.05, 2.0, 30)
    dvals = np.linspace(0.5, 2.0, 30)       # operator A = diag(lam * dvals), D = diag(dvals)
    Adiag = lam * dvals
    r = synthetic.uniform_vector(30, 4)
    lo, hi = 0.1, 2.2
    z = fem.chebyshev(lambda v: Adiag * v, 1.0 / dvals, r, degree, lo, hi)
    # closed form p(lambda) = (1 - T_m(sigma(lambda)) / T_m(sigma(0))) / lambda,  z = p(D^-1 A) D^-1 r
    T = np.polynomial.chebyshev.Chebyshev.basis(degree)
    sig = lambda l: (hi + lo - 2 * l) / (hi - lo)
    p = (1.0 - T(sig(lam)) / T(sig(0.0))) / lam
    assert np.allclose(z, p * r / dvals, atol=1e-13)


def test_lanczos_estimate_matches_dense_eigenvalue():
    m = mesh.structured_mesh(3, 3, 3, 2)
    K = fem.assemble(m, 3)
    d = fem.diagonal(K)
    lam_true = np.linalg.eigvals(np.diag(1 / d) @ K.toarray()).real.max()
    start = synthetic.uniform_vector(m.n_dofs, 5)
    est = fem.lanczos_lambda_max(lambda v: K @ v, 1 / d, start, steps=40)
    assert est <= lam_true * (1 + 1e-10)
    assert est > 0.98 * lam_true
    est15 = fem.lanczos_lambda_max(lambda v: K @ v, 1 / d, start, steps=15)
    assert 0.8 * lam_true < est15 <= lam_true * (1 + 1e-10)


def test_defect_correction_reaches_fp64_solution():
    m = mesh.structured_mesh(4, 4, 4, 3, synthetic.deformed_vertices(4, 4, 4))
    K = fem.assemble(m, 4, fem.COEF_TRIG, (1.0, 0.5))
    K32 = K.astype(np.float32)
    b = synthetic.gaussian_vector(m.n_dofs, 6)
    b[m.constrained] = 0
    d = fem.diagonal(K)
    lmax = fem.lanczos_lambda_max(lambda v: K @ v, 1 / d, synthetic.uniform_vector(m.n_dofs, 7), 15)
    hi, lo = 1.2 * lmax, 1.2 * lmax / 20
    d32 = (1 / d).astype(np.float32)
    prec = lambda r: fem.chebyshev(lambda v: K32 @ v, d32, r, 5, lo, hi, dtype=np.float32)
    res = fem.defect_correction(lambda v: K @ v, lambda v: K32 @ v, 1 / d, b, prec, tol=1e-10, inner_tol=1e-4)
    assert res.status == 0
    assert np.linalg.norm(b - K @ res.x) <= 1e-10 * np.linalg.norm(b)
    xd = spla.spsolve(K.tocsc(), b)
    assert np.linalg.norm(res.x - xd) < 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("kind", ["structured", "octree"])
def test_pure_neumann_operator_annihilates_constants(kind):
    """With no Dirichlet face the weak Laplacian of a constant vanishes for any geometry and coefficient:
    C^T A C applied to the constant free vector is zero (hanging interpolation reproduces constants)."""
    if kind == "structured":
        m = mesh.structured_mesh(3, 3, 2, 2, synthetic.deformed_vertices(3, 3, 2), dirichlet=0)
        assert len(m.constrained) == 0
    else:
        leaves = synthetic.octree_leaves(3, 1, np.array([0.3, 0.4, 0.5]), 0.3)
        m = mesh.octree_mesh(3, 3, 3, 2, leaves, synthetic.deformed_vertices(3, 3, 3), dirichlet=0)
        assert len(m.constrained) > 0 and all(m.cptr[1:] > m.cptr[:-1])  # hanging rows only
    K = fem.assemble(m, 3, fem.COEF_TRIG, (1.0, 0.5))
    v = np.ones(m.n_dofs)
    v[m.constrained] = 0.0
    r = K @ v
    assert np.abs(r).max() < 1e-12 * abs(K).max()
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_mixed_boundary_manufactured_convergence(k):
    """Dirichlet on the x faces only, natural boundaries elsewhere: u = sin(pi x) solves -lap u = pi^2 sin(pi x)
    with zero normal derivative on the y and z faces (the deformation keeps every face of the box in
    place), so the L2 error falls at the optimal rate k + 1."""
    sizes = (2, 4, 8) if k < 3 else (2, 4, 6)
    errs = []
    for nx in sizes:
        m = mesh.structured_mesh(nx, nx, nx, k, synthetic.deformed_vertices(nx, nx, nx), dirichlet=0b11)
        X, _ = fem.quadrature_points(m, k + 1)
        fq = np.pi ** 2 * np.sin(np.pi * X[..., 0])
        K = fem.assemble(m, k + 1)
        x = spla.spsolve(K.tocsc(), fem.rhs(m, k + 1, fq=fq))
        errs.append(fem.l2_error(m, x, exact="sinx"))
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(sizes[i + 1] / sizes[i]) for i in range(len(errs) - 1)]
    assert rates[-1] > k + 1 - 0.35, (errs, rates)
