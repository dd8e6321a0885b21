"""Pins of the oracle's multigrid cycle (oracle/mg.py) against what the mathematics fixes."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, mg
from oracle.rules import gauss_lobatto
from paper_1910_13247_gb300 import synthetic


def logical_coords(n_cells, k):
    """Logical coordinate in [0, 1] of every lattice point of one direction (cell-wise GLL nodes)."""
    x = gauss_lobatto(k)
    M = k * n_cells + 1
    out = np.zeros(M)
    for I in range(M):
        c = min(I // k, n_cells - 1)
        out[I] = (c + x[I - c * k]) / n_cells
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prolongation_reproduces_tensor_polynomials(k):
    """P applied to the coarse interpolant of a Q_k polynomial (in logical coordinates) gives the
    polynomial at the fine nodes exactly: the coarse cell's Q_k interpolant reproduces it."""
    nc = (3, 2, 2)
    sizes = [nc, tuple(2 * s for s in nc)]
    meshes = [mg.structured_mesh(*s, k) for s in sizes]
    P = mg.prolongation(meshes[0], meshes[1], nc, k, condensed=False)
    rng = np.random.default_rng(k)
    coef = rng.uniform(-1, 1, (k + 1, k + 1, k + 1))

    def values(size):
        X, Y, Z = (logical_coords(s, k) for s in size)
        px = np.vander(X, k + 1, increasing=True)
        py = np.vander(Y, k + 1, increasing=True)
        pz = np.vander(Z, k + 1, increasing=True)
        return np.einsum("abc,la,jb,ic->ijl", coef, px, py, pz).ravel()  # (L, J, I) order: x fastest

    uc, uf = values(sizes[0]), values(sizes[1])
    assert np.abs(P @ uc - uf).max() < 1e-13 * np.abs(uf).max()
    # rows are partitions of unity
    assert np.abs(np.asarray(P.sum(axis=1)).ravel() - 1.0).max() < 1e-14


def test_level_sizes_and_coarse_vertices():
    assert mg.level_sizes(96, 96, 96) == [(3, 3, 3), (6, 6, 6), (12, 12, 12), (24, 24, 24), (48, 48, 48), (96, 96, 96)]
    assert mg.level_sizes(64, 64, 64)[0] == (1, 1, 1) and len(mg.level_sizes(64, 64, 64)) == 7
    assert mg.level_sizes(128, 64, 64)[0] == (2, 1, 1) and len(mg.level_sizes(128, 64, 64)) == 7
    assert mg.level_sizes(8, 8, 6) == [(4, 4, 3), (8, 8, 6)]
    assert mg.level_sizes(16, 16, 16, max_levels=2) == [(8, 8, 8), (16, 16, 16)]
    v = synthetic.deformed_vertices(4, 4, 4)
    vc = mg.coarsen_vertices(v, 4, 4, 4)
    assert vc.shape == (27, 3) and np.array_equal(vc[13], v.reshape(5, 5, 5, 3)[2, 2, 2])


def _hier(n, k, levels=0, degree=4):
    meshes, sizes = mg.level_meshes(n, n, n, k, synthetic.deformed_vertices(n, n, n), max_levels=levels)
    return mg.Hierarchy(meshes, sizes, k, fem.COEF_TRIG, (1.0, 0.5), degree=degree)


def test_single_level_cycle_is_the_exact_inverse():
    h = _hier(4, 2, levels=1)
    b = synthetic.uniform_vector(h.meshes[0].n_dofs, 3)
    z = h.vcycle(b)
    K = h.K[0]
    assert np.linalg.norm(K @ z - b) < 1e-12 * np.linalg.norm(b)


def test_vcycle_is_symmetric_and_positive():
    h = _hier(8, 2)
    assert len(h.meshes) == 4
    n = h.meshes[-1].n_dofs
    x, y = synthetic.uniform_vector(n, 4), synthetic.uniform_vector(n, 5)
    vx, vy = h.vcycle(x), h.vcycle(y)
    assert abs(y @ vx - x @ vy) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * 10
    assert x @ vx > 0 and y @ vy > 0


def test_mg_pcg_iterations_do_not_grow_with_the_mesh():
    """The V-cycle is a uniformly good preconditioner: PCG iterations to 1e-10 stay bounded and do
    not grow with refinement (Jacobi-PCG iterations double with each refinement)."""
    its = []
    for n in (4, 8, 16):
        h = _hier(n, 2)
        K = h.K[-1]
        b = synthetic.uniform_vector(K.shape[0], 6)
        b[h.meshes[-1].constrained] = 0.0
        res = fem.pcg(lambda v: K @ v, b, h.vcycle, tol=1e-10)
        assert res.status == 0
        assert np.linalg.norm(b - K @ res.x) <= 1.0001e-10 * np.linalg.norm(b)
        its.append(res.iterations)
    assert max(its) <= 15 and its[2] <= its[1] + 2, its
    jac = fem.pcg(lambda v: K @ v, b, lambda r: r / fem.diagonal(K), tol=1e-10)
    assert jac.iterations > 3 * its[2]
