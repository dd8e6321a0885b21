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
