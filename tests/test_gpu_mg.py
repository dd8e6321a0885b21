"""Geometric multigrid (mfx_mg_*): the V-cycle equals the oracle's cycle (oracle/mg.py) built with the
same smoother intervals, the hierarchy has the oracle's levels, and MG-preconditioned PCG (FP64 and
mixed precision) reaches the 1e-10 residual in the oracle's iteration counts, independently of the mesh."""
import numpy as np
import pytest

from oracle import fem, mg as omg
from paper_1910_13247_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mfx():
    from paper_1910_13247_gb300 import build, mfx as m
    build.build()
    m.lib()
    return m


def make(mfx, n, k, faces=0x3F, degree=4):
    verts = synthetic.deformed_vertices(n, n, n)
    mesh = mfx.Mesh.structured_box(n, n, n, verts, dirichlet=faces)
    g = mfx.Multigrid(mesh, k, mfx.COEF_TRIG, (1.0, 0.5), smoother_degree=degree)
    meshes, sizes = omg.level_meshes(n, n, n, k, verts, dirichlet=faces)
    assert g.n_levels == len(meshes)
    bounds = [None] + [g.bounds(l) for l in range(1, g.n_levels)]
    h = omg.Hierarchy(meshes, sizes, k, fem.COEF_TRIG, (1.0, 0.5), degree=degree,
                      bounds=[(1.0, 2.0)] + bounds[1:])
    # the library's Lanczos intervals agree with the oracle's own estimates
    h2 = omg.Hierarchy(meshes[-2:], sizes[-2:], k, fem.COEF_TRIG, (1.0, 0.5), degree=degree)
    lo, hi = g.bounds(g.n_levels - 1)
    assert abs(hi - h2.bounds[-1][1]) < 1e-6 * hi
    return g, h, meshes


@pytest.mark.parametrize("n,k,faces", [(8, 2, 0x3F), (8, 3, 0x3F), (12, 2, 0x3F), (8, 4, 0b000011), (4, 1, 0x3F)])
def test_vcycle_equals_the_oracle_cycle(mfx, n, k, faces):
    g, h, meshes = make(mfx, n, k, faces)
    assert g.coarse_free_dofs == int(h.free[0].sum())
    r = synthetic.uniform_vector(meshes[-1].n_dofs, 70 + k)
    ref = h.vcycle(r)
    z = torch.empty(meshes[-1].n_dofs, dtype=torch.float64, device=DEV)
    g.vcycle(torch.tensor(r, device=DEV), z)
    zz = z.cpu().numpy()
    assert np.linalg.norm(zz - ref) < 1e-10 * np.linalg.norm(ref), np.linalg.norm(zz - ref) / np.linalg.norm(ref)
    z32 = torch.empty(meshes[-1].n_dofs, dtype=torch.float32, device=DEV)
    g.vcycle(torch.tensor(r, device=DEV).float(), z32)
    assert np.linalg.norm(z32.cpu().double().numpy() - ref) < 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("mixed", [False, True])
def test_mg_pcg_matches_oracle_iterations_and_residual(mfx, mixed):
    its = []
    for n in (8, 16):
        g, h, meshes = make(mfx, n, 2)
        K = h.K[-1]
        b = synthetic.uniform_vector(meshes[-1].n_dofs, 80)
        b[meshes[-1].constrained] = 0.0
        x = torch.zeros(meshes[-1].n_dofs, dtype=torch.float64, device=DEV)
        st = g.solve(torch.tensor(b, device=DEV), x, tol=1e-10, mixed=mixed)
        assert st["status"] == 0
        xs = x.cpu().numpy()
        assert np.linalg.norm(b - K @ xs) <= 1.0001e-10 * np.linalg.norm(b)
        if not mixed:
            ref = fem.pcg(lambda v: K @ v, b, h.vcycle, tol=1e-10)
            assert abs(st["iterations"] - ref.iterations) <= 1, (st["iterations"], ref.iterations)
            assert np.linalg.norm(xs - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
            its.append(st["iterations"])
    if its:
        assert max(its) <= 12 and its[1] <= its[0] + 2, its


def test_mg_options_and_errors(mfx):
    verts = synthetic.deformed_vertices(8, 8, 8)
    mesh = mfx.Mesh.structured_box(8, 8, 8, verts)
    g = mfx.Multigrid(mesh, 2, mfx.COEF_TRIG, (1.0, 0.5), max_levels=2)
    assert g.n_levels == 2
    lo, hi = g.bounds(1)
    g.set_bounds(1, lo / 2, hi)
    assert g.bounds(1) == (lo / 2, hi)
    # the cycle with the new interval equals the oracle's with the same interval
    meshes, sizes = omg.level_meshes(8, 8, 8, 2, verts, max_levels=2)
    h = omg.Hierarchy(meshes, sizes, 2, fem.COEF_TRIG, (1.0, 0.5), degree=6, bounds=[(1.0, 2.0), (lo / 2, hi)])
    r = synthetic.uniform_vector(meshes[-1].n_dofs, 90)
    z = torch.empty(meshes[-1].n_dofs, dtype=torch.float64, device=DEV)
    g.vcycle(torch.tensor(r, device=DEV), z)
    ref = h.vcycle(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) < 1e-10 * np.linalg.norm(ref)
    with pytest.raises(mfx.MfxError):
        g.set_bounds(0, 1.0, 2.0)  # the coarsest level has no smoother
    leaves = synthetic.octree_leaves(2, 1, np.array([0.5, 0.5, 0.5]), 0.3)
    with pytest.raises(mfx.MfxError) as e:
        mfx.Multigrid(mfx.Mesh.octree(2, 2, 2, leaves), 2)
    assert e.value.code == mfx.EUNSUPPORTED
