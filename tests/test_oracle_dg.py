"""Pins of the oracle's SIPG operator (oracle/dg.py) against what the mathematics fixes."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import dg, fem
from oracle import mesh as omesh


def test_symmetric_positive_definite():
    K = dg.dg_operator(2, 2, 2, 2).toarray()
    assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_pure_neumann_operator_annihilates_constants(k):
    """Without Dirichlet faces every face term of a constant vanishes (no jumps, no gradients)."""
    K = dg.dg_operator(3, 2, 2, k, lengths=(1.0, 0.5, 2.0), dirichlet=0)
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-11 * abs(K).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_equals_the_continuous_form_on_continuous_functions(k):
    """For continuous functions vanishing on the boundary all face terms vanish, so the SIPG form is
    the continuous Galerkin form (checked against the pinned CG assembly through the injection)."""
    nx, ny, nz = 3, 2, 2
    cg = omesh.structured_mesh(nx, ny, nz, k)
    Kc = fem.assemble(cg, k + 1)
    P = dg.injection(cg, k)
    Kd = dg.dg_operator(nx, ny, nz, k)
    rng = np.random.default_rng(k)
    u, v = rng.uniform(-1, 1, cg.n_dofs), rng.uniform(-1, 1, cg.n_dofs)
    u[cg.constrained] = 0.0
    v[cg.constrained] = 0.0
    lhs = (P @ u) @ (Kd @ (P @ v))
    rhs = u @ (Kc @ v)
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(v) * abs(Kc).max()


@pytest.mark.parametrize("k,sizes", [(1, (2, 4, 8)), (2, (2, 4, 8)), (3, (2, 4))])
def test_manufactured_convergence_rate(k, sizes):
    """u = sin(pi x) sin(pi y) sin(pi z) (zero on the boundary, imposed weakly): optimal L2 rate k + 1."""
    errs = []
    for n in sizes:
        K = dg.dg_operator(n, n, n, k)
        m = dg.dg_mesh(n, n, n, k)
        X, _ = fem.quadrature_points(m, k + 1)
        fq = 3 * np.pi ** 2 * np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
        x = spla.spsolve(K.tocsc(), fem.rhs(m, k + 1, fq=fq))
        errs.append(fem.l2_error(m, x))
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(sizes[i + 1] / sizes[i]) for i in range(len(errs) - 1)]
    assert rates[-1] > k + 1 - 0.35, (errs, rates)


def test_multigrid_with_a_discontinuous_top_level():
    """SIPG on top of the continuous hierarchy (injection, then h-coarsening): a symmetric cycle that
    makes PCG converge in a few iterations, independently of the mesh."""
    from oracle import mg
    its = []
    for n in (4, 8):
        k = 2
        meshes, sizes = mg.level_meshes(n, n, n, k)
        Kd = dg.dg_operator(n, n, n, k)
        h = mg.Hierarchy(meshes, sizes, k, degree=6, dg_top=(Kd, dg.injection(meshes[-1], k)))
        x = np.random.default_rng(1).uniform(-1, 1, Kd.shape[0])
        y = np.random.default_rng(2).uniform(-1, 1, Kd.shape[0])
        assert abs(y @ h.vcycle(x) - x @ h.vcycle(y)) < 1e-11 * np.linalg.norm(x) * np.linalg.norm(y)
        res = fem.pcg(lambda v: Kd @ v, x, h.vcycle, tol=1e-10)
        assert res.status == 0
        its.append(res.iterations)
    assert max(its) <= 20 and its[1] <= its[0] + 3, its


def _sipg_1d_k1(nc, h, eta, dir_lo, dir_hi):
    """1D SIPG matrix of linear elements on nc cells of size h, written out by hand from the 1D form
    sum_c int u'v' + sum_interior (-{u'}[v] - [u]{v'} + s [u][v]) + Dirichlet ends (-u'_n v - u v'_n + s_b u v),
    s = eta (k+1)^2 / h = 4 eta / h, s_b = 2 s.  DoFs (cell, local node), the cell's node 0 at its left end."""
    from fractions import Fraction as F
    n = 2 * nc
    A = [[F(0)] * n for _ in range(n)]
    hh, s = F(h), 4 * F(eta) / F(h)
    # basis of cell c: phi_0 = 1 - t, phi_1 = t on x = (c + t) h; values at t = 0, 1 and the slope
    val = {0: (1, 0), 1: (0, 1)}          # val[node] = (value at left end, value at right end)
    slope = {0: -1 / hh, 1: 1 / hh}
    for c in range(nc):
        for i in range(2):
            for j in range(2):
                A[2 * c + i][2 * c + j] += slope[i] * slope[j] * hh
    for c in range(nc - 1):  # face between cell c ("-") and c + 1 ("+")
        for a in range(2):
            for b in range(2):
                for ca, cb in ((c, c), (c, c + 1), (c + 1, c), (c + 1, c + 1)):
                    ja = val[a][1] if ca == c else -val[a][0]      # jump of test function
                    jb = val[b][1] if cb == c else -val[b][0]      # jump of trial function
                    aa = slope[a] / 2                               # average of derivatives
                    ab = slope[b] / 2
                    A[2 * ca + a][2 * cb + b] += -ab * ja - jb * aa + s * ja * jb
    for end, on in ((0, dir_lo), (1, dir_hi)):
        if not on:
            continue
        c = 0 if end == 0 else nc - 1
        sign = -1 if end == 0 else 1                                # outward normal
        for a in range(2):
            for b in range(2):
                va, vb = val[a][end], val[b][end]
                A[2 * c + a][2 * c + b] += -sign * slope[b] * va - sign * slope[a] * vb + 2 * s * va * vb
    return np.array([[float(x) for x in row] for row in A])


def _mass_1d_k1(nc, h):
    m = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]]) * h
    return np.kron(np.eye(nc), m)


def test_box_operator_is_the_kronecker_sum_of_1d_sipg_matrices():
    """On a uniform box with a constant coefficient the SIPG form separates: A = a sum_d L_d (x) M (x) M
    with the 1D SIPG and mass matrices of each direction (written out above by hand for k = 1, with the
    penalty eta (k+1)^2 / h of the reading); the oracle's 3D full-quadrature matrix must equal it, per
    direction with its own cell size and its own Dirichlet ends."""
    nx, ny, nz, k = 3, 2, 2, 1
    L = (1.5, 1.0, 0.5)
    faces = 0b011101  # x: both ends, y: high end only, z: low end only
    eta, coef = 1.7, 0.9
    K = dg.dg_operator(nx, ny, nz, k, L, faces, eta=eta, coef=coef).toarray()
    dims, h = (nx, ny, nz), [L[d] / (nx, ny, nz)[d] for d in range(3)]
    Ls = [_sipg_1d_k1(dims[d], h[d], eta, bool(faces >> (2 * d) & 1), bool(faces >> (2 * d + 1) & 1)) for d in range(3)]
    Ms = [_mass_1d_k1(dims[d], h[d]) for d in range(3)]
    # tensor index (z slowest): flat_d = c_d * 2 + i_d
    T = coef * (np.kron(Ms[2], np.kron(Ms[1], Ls[0])) + np.kron(Ms[2], np.kron(Ls[1], Ms[0])) +
                np.kron(Ls[2], np.kron(Ms[1], Ms[0])))
    # cell-major order of the oracle: cell (x fastest) * 8 + local (i1 + 2 i2 + 4 i3)
    perm = np.zeros(T.shape[0], dtype=np.int64)
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                for i3 in range(2):
                    for i2 in range(2):
                        for i1 in range(2):
                            g = ((cz * ny + cy) * nx + cx) * 8 + i1 + 2 * i2 + 4 * i3
                            t = ((cz * 2 + i3) * (2 * ny) + cy * 2 + i2) * (2 * nx) + cx * 2 + i1
                            perm[g] = t
    Tg = T[np.ix_(perm, perm)]
    assert np.abs(K - Tg).max() < 1e-12 * np.abs(K).max()
