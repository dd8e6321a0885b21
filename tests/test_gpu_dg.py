"""SIPG operator (discretization = SIPG): vmult and diagonal equal the oracle's assembled SIPG matrix
(oracle/dg.py) element by element, FP64 within 1e-12 and FP32 within 1e-5 (relative to the largest
entry), for every compiled degree, anisotropic cells and every kind of face mask; PCG on the DG operator
solves its system; the multigrid hierarchy with the SIPG level on top equals the oracle's cycle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import dg as odg, fem, mg as omg
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


def box(dims, lengths):
    return synthetic.lattice_vertices(*dims) * np.asarray(lengths)[None, :]


def sipg(mfx, dims, k, lengths=(1.0, 1.0, 1.0), faces=0x3F, eta=1.0, coef=1.0, precisions=3):
    mesh = mfx.Mesh.structured_box(*dims, box(dims, lengths), dirichlet=faces)
    return mfx.Operator(mesh, k, mfx.COEF_CONSTANT, (coef, 0.0), precisions=precisions, discretization=mfx.SIPG,
                        dg_penalty=eta)


def apply(op, x, dtype):
    src = torch.tensor(x, device=DEV, dtype=dtype)
    dst = torch.empty_like(src)
    op.vmult(src, dst)
    return dst.cpu().double().numpy()


CASES = [
    ((3, 2, 4), 1, (1.0, 1.0, 1.0), 0x3F, 1.0, 1.0),
    ((3, 3, 2), 2, (1.0, 0.7, 1.3), 0x3F, 1.5, 0.8),
    ((2, 3, 2), 3, (1.0, 1.0, 1.0), 0b010110, 1.0, 1.0),
    ((3, 2, 2), 4, (2.0, 1.0, 1.0), 0, 2.0, 1.0),
    ((2, 2, 3), 5, (1.0, 1.0, 1.0), 0b101001, 1.0, 3.0),
    ((2, 2, 2), 6, (1.0, 0.5, 1.0), 0x3F, 1.0, 1.0),
    ((2, 1, 2), 7, (1.0, 1.0, 1.0), 0b001100, 1.0, 1.0),
    ((2, 2, 1), 8, (1.0, 1.0, 0.5), 0b100001, 1.0, 1.0),
]


@pytest.mark.parametrize("dims,k,lengths,faces,eta,coef", CASES)
def test_sipg_vmult_and_diagonal_equal_the_oracle(mfx, dims, k, lengths, faces, eta, coef):
    K = odg.dg_operator(*dims, k, lengths, faces, eta=eta, coef=coef)
    op = sipg(mfx, dims, k, lengths, faces, eta, coef)
    info = op.info()
    assert op.n_dofs == K.shape[0] and info["discretization"] == mfx.SIPG and info["n_constrained"] == 0
    x = synthetic.uniform_vector(op.n_dofs, 300 + k)
    ref = K @ x
    scale = np.abs(ref).max()
    y = apply(op, x, torch.float64)
    assert np.abs(y - ref).max() <= 1e-12 * scale, np.abs(y - ref).max() / scale
    y32 = apply(op, x, torch.float32)
    assert np.abs(y32 - ref).max() <= 1e-5 * scale, np.abs(y32 - ref).max() / scale
    d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.diagonal(d)
    dref = K.diagonal()
    assert np.abs(d.cpu().numpy() - dref).max() <= 1e-12 * np.abs(dref).max()
    d32 = torch.empty(op.n_dofs, dtype=torch.float32, device=DEV)
    op.diagonal(d32)
    assert np.abs(d32.cpu().double().numpy() - dref).max() <= 1e-6 * np.abs(dref).max()
    # cell-major DoFs, nothing constrained
    t = op.tables()
    assert np.array_equal(t["cell_dofs"].ravel(), np.arange(op.n_dofs)) and t["constrained"].size == 0


@pytest.mark.parametrize("k,dims", [(1, (9, 8, 5)), (2, (7, 5, 3)), (3, (7, 5, 4)), (4, (7, 5, 3)), (5, (6, 5, 3)),
                                    (6, (5, 3, 2))])
def test_sipg_many_cells_span_several_blocks_and_a_ragged_tail(mfx, k, dims):
    """More cells than one CTA batch, batches that start inside a row of cells and whose y and z
    neighbours lie in other batches, and a partial last batch; FP64 and FP32 (the FP32 plane kernel at
    degrees 1..5, the line kernel at 6) against the oracle matrix."""
    K = odg.dg_operator(*dims, k, (1.0, 1.2, 0.9), 0b011011)
    op = sipg(mfx, dims, k, (1.0, 1.2, 0.9), 0b011011)
    x = synthetic.uniform_vector(op.n_dofs, 41)
    ref = K @ x
    scale = np.abs(ref).max()
    y = apply(op, x, torch.float64)
    assert np.abs(y - ref).max() <= 1e-12 * scale
    y32 = apply(op, x, torch.float32)
    assert np.abs(y32 - ref).max() <= 1e-5 * scale, np.abs(y32 - ref).max() / scale


@pytest.mark.parametrize("k,dims,faces", [(1, (1, 1, 1), 0x3F), (3, (1, 1, 1), 0b100110), (5, (1, 1, 1), 0),
                                          (2, (1, 5, 7), 0x3F), (4, (6, 1, 4), 0b011001), (3, (5, 4, 1), 0x3F),
                                          (4, (1, 30, 2), 0b110011), (2, (27, 1, 1), 0b000011)])
def test_sipg_fp32_degenerate_boxes(mfx, k, dims, faces):
    """Boxes one cell thick in some direction (no neighbours there; a batch of the FP32 plane kernel spans
    several rows or planes of cells, and its staged neighbour chunks overlap its own), a single cell, and
    natural faces: FP32 against the oracle matrix."""
    K = odg.dg_operator(*dims, k, (1.0, 0.8, 1.1), faces)
    op = sipg(mfx, dims, k, (1.0, 0.8, 1.1), faces)
    x = synthetic.uniform_vector(op.n_dofs, 47 + k)
    ref = K @ x
    scale = np.abs(ref).max()
    y32 = apply(op, x, torch.float32)
    assert np.abs(y32 - ref).max() <= 1e-5 * scale, np.abs(y32 - ref).max() / scale


@pytest.mark.parametrize("k", [2, 4])
def test_sipg_fp32_source_not_16_byte_aligned(mfx, k):
    """A source vector that starts 4 bytes past a 16-byte boundary takes the FP32 line kernel (the plane
    kernel stages with 16-byte loads); both give the oracle's product."""
    dims = (7, 5, 3)
    K = odg.dg_operator(*dims, k, (1.0, 1.2, 0.9), 0b011011)
    op = sipg(mfx, dims, k, (1.0, 1.2, 0.9), 0b011011)
    x = synthetic.uniform_vector(op.n_dofs, 43)
    ref = K @ x
    buf = torch.zeros(op.n_dofs + 1, dtype=torch.float32, device=DEV)
    src = buf[1:]
    src.copy_(torch.tensor(x, dtype=torch.float32, device=DEV))
    assert src.data_ptr() % 16 == 4
    dst = torch.empty_like(src)
    op.vmult(src, dst)
    y32 = dst.cpu().double().numpy()
    assert np.abs(y32 - ref).max() <= 1e-5 * np.abs(ref).max()


def test_sipg_pure_neumann_kernel_is_the_constants(mfx):
    """Without Dirichlet faces the SIPG form vanishes on constants (no jumps, no gradients)."""
    op = sipg(mfx, (3, 3, 3), 3, faces=0)
    one = np.ones(op.n_dofs)
    y = apply(op, one, torch.float64)
    x = synthetic.uniform_vector(op.n_dofs, 5)
    assert np.abs(y).max() <= 1e-12 * np.abs(apply(op, x, torch.float64)).max()


def test_sipg_pcg_solves_the_system(mfx):
    dims, k = (4, 4, 4), 2
    K = odg.dg_operator(*dims, k)
    op = sipg(mfx, dims, k)
    b = synthetic.uniform_vector(op.n_dofs, 9)
    x = torch.zeros(op.n_dofs, dtype=torch.float64, device=DEV)
    st = op.solve(torch.tensor(b, device=DEV), x, tol=1e-10, precond=mfx.PRECOND_CHEBYSHEV, cheb_degree=4)
    assert st["status"] == 0
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - K @ xs) <= 1.0001e-10 * np.linalg.norm(b)
    ref = spla.spsolve(K.tocsc(), b)
    assert np.linalg.norm(xs - ref) <= 1e-7 * np.linalg.norm(ref)


def test_sipg_rejects_what_it_does_not_cover(mfx):
    v = synthetic.deformed_vertices(3, 3, 3)
    mesh = mfx.Mesh.structured_box(3, 3, 3, v)
    with pytest.raises(mfx.MfxError) as e:
        mfx.Operator(mesh, 2, discretization=mfx.SIPG)
    assert e.value.code == mfx.EUNSUPPORTED
    mesh = mfx.Mesh.structured_box(3, 3, 3, box((3, 3, 3), (1, 1, 1)))
    with pytest.raises(mfx.MfxError) as e:
        mfx.Operator(mesh, 2, mfx.COEF_TRIG, (1.0, 0.5), discretization=mfx.SIPG)
    assert e.value.code == mfx.EUNSUPPORTED
    op = mfx.Operator(mesh, 2, discretization=mfx.SIPG)
    b = torch.zeros(op.n_dofs, dtype=torch.float64, device=DEV)
    op.distribute(b)  # nothing constrained: a no-op
    assert float(b.abs().max()) == 0.0


def test_sipg_poisson_solve_equals_the_oracle_solution(mfx):
    """A manufactured Poisson problem solved with the SIPG operator: quadrature points and load vector
    equal the oracle's, the MG-PCG solution equals the oracle's direct solution, and the L2 error
    (the oracle's routine) falls at the optimal rate k + 1 under refinement."""
    k, errs = 2, []
    for n in (4, 8):
        verts = box((n, n, n), (1.0, 1.0, 1.0))
        mesh = mfx.Mesh.structured_box(n, n, n, verts)
        g = mfx.Multigrid(mesh, k, smoother_degree=6, discretization=mfx.SIPG)
        op = g.fine
        n3 = (k + 1) ** 3
        om = odg.dg_mesh(n, n, n, k)
        X, _ = fem.quadrature_points(om, k + 1)
        xq = torch.empty(om.cell_dofs.shape[0] * n3 * 3, dtype=torch.float64, device=DEV)
        op.quadrature_points(xq)
        assert np.abs(xq.cpu().numpy().reshape(X.shape) - X).max() < 1e-14
        fq = 3 * np.pi ** 2 * np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
        b_ref = fem.rhs(om, k + 1, fq=fq)
        b = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
        op.rhs(torch.tensor(fq.ravel(), device=DEV), b)
        assert np.abs(b.cpu().numpy() - b_ref).max() <= 1e-13 * np.abs(b_ref).max()
        b2 = torch.empty_like(b)  # the same load vector from a host function
        op.rhs_function(lambda x, y, z: 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z), b2)
        assert np.abs(b2.cpu().numpy() - b_ref).max() <= 1e-13 * np.abs(b_ref).max()
        x = torch.zeros_like(b)
        st = g.solve(b, x, tol=1e-12)
        assert st["status"] == 0
        K = odg.dg_operator(n, n, n, k)
        x_ref = spla.spsolve(K.tocsc(), b_ref)
        xs = x.cpu().numpy()
        assert np.linalg.norm(xs - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
        errs.append(fem.l2_error(om, xs))
    rate = np.log2(errs[0] / errs[1])
    assert rate > k + 1 - 0.35, (errs, rate)


def dg_hierarchy(mfx, n, k, faces, degree=4, lengths=(1.0, 1.0, 1.0)):
    verts = box((n, n, n), lengths)
    mesh = mfx.Mesh.structured_box(n, n, n, verts, dirichlet=faces)
    g = mfx.Multigrid(mesh, k, mfx.COEF_CONSTANT, (1.0, 0.0), smoother_degree=degree, discretization=mfx.SIPG)
    meshes, sizes = omg.level_meshes(n, n, n, k, verts, dirichlet=faces)
    assert g.n_levels == len(meshes) + 1
    Kdg = odg.dg_operator(n, n, n, k, lengths, faces)
    P = odg.injection(meshes[-1], k)
    bounds = [(1.0, 2.0)] + [g.bounds(l) for l in range(1, g.n_levels)]
    h = omg.Hierarchy(meshes, sizes, k, fem.COEF_CONSTANT, (1.0, 0.0), degree=degree, bounds=bounds,
                      dg_top=(Kdg, P))
    # the library's Lanczos interval of the SIPG level agrees with the oracle's own estimate
    h2 = omg.Hierarchy(meshes[-1:], sizes[-1:], k, fem.COEF_CONSTANT, (1.0, 0.0), degree=degree, dg_top=(Kdg, P))
    lo, hi = g.bounds(g.n_levels - 1)
    assert abs(hi - h2.bounds[-1][1]) < 1e-6 * hi
    return g, h, Kdg


@pytest.mark.parametrize("n,k,faces", [(8, 2, 0x3F), (4, 3, 0x3F), (8, 1, 0b001111), (4, 4, 0x3F)])
def test_sipg_multigrid_vcycle_equals_the_oracle_cycle(mfx, n, k, faces):
    g, h, Kdg = dg_hierarchy(mfx, n, k, faces)
    assert g.fine.info()["discretization"] == mfx.SIPG
    r = synthetic.uniform_vector(Kdg.shape[0], 90 + k)
    ref = h.vcycle(r)
    z = torch.empty(Kdg.shape[0], dtype=torch.float64, device=DEV)
    g.vcycle(torch.tensor(r, device=DEV), z)
    zz = z.cpu().numpy()
    assert np.linalg.norm(zz - ref) < 1e-10 * np.linalg.norm(ref), np.linalg.norm(zz - ref) / np.linalg.norm(ref)
    z32 = torch.empty(Kdg.shape[0], dtype=torch.float32, device=DEV)
    g.vcycle(torch.tensor(r, device=DEV).float(), z32)
    assert np.linalg.norm(z32.cpu().double().numpy() - ref) < 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("mixed", [False, True])
def test_sipg_multigrid_pcg_matches_the_oracle(mfx, mixed):
    g, h, Kdg = dg_hierarchy(mfx, 8, 2, 0x3F)
    b = synthetic.uniform_vector(Kdg.shape[0], 95)
    x = torch.zeros(Kdg.shape[0], dtype=torch.float64, device=DEV)
    st = g.solve(torch.tensor(b, device=DEV), x, tol=1e-10, mixed=mixed)
    assert st["status"] == 0
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - Kdg @ xs) <= 1.0001e-10 * np.linalg.norm(b)
    if not mixed:
        ref = fem.pcg(lambda v: Kdg @ v, b, h.vcycle, tol=1e-10)
        assert abs(st["iterations"] - ref.iterations) <= 1, (st["iterations"], ref.iterations)
        assert st["iterations"] <= 15


def test_sipg_full_size_sampled_rows(mfx):
    """The benchmark's SIPG workload at full size (p = 4, 128 x 64 x 64 cells of [0,2] x [0,1] x [0,1],
    65.5M DoFs) in the benchmark's launch configuration: the rows of sampled cells against the oracle.
    A cell's rows involve only the cell and its face neighbours, so the oracle's matrix of the sub-box of
    the cell and its neighbours (same cell size; the box's own faces where the sub-box touches them)
    gives them exactly; corner, edge, face and interior cells are sampled."""
    dims, k, lengths, faces = (128, 64, 64), 4, (2.0, 1.0, 1.0), 0x3F
    n3 = (k + 1) ** 3
    op = sipg(mfx, dims, k, lengths, faces)
    n = op.n_dofs
    gen = torch.Generator(device=DEV).manual_seed(71)
    x = torch.rand(n, generator=gen, dtype=torch.float64, device=DEV) * 2 - 1
    y = torch.empty_like(x)
    op.vmult(x, y)
    x32 = x.float()
    y32 = torch.empty_like(x32)
    op.vmult(x32, y32)
    h = [lengths[d] / dims[d] for d in range(3)]
    samples = [(0, 0, 0), (127, 63, 63), (0, 31, 63), (64, 0, 17), (5, 63, 40), (77, 12, 0), (100, 50, 33),
               (1, 1, 1)]
    for c in samples:
        lo = [max(0, c[d] - 1) for d in range(3)]
        hi = [min(dims[d] - 1, c[d] + 1) for d in range(3)]
        sd = [hi[d] - lo[d] + 1 for d in range(3)]
        mask = 0
        for d in range(3):
            if lo[d] > 0 or (faces >> (2 * d)) & 1:
                mask |= 1 << (2 * d)
            if hi[d] < dims[d] - 1 or (faces >> (2 * d + 1)) & 1:
                mask |= 1 << (2 * d + 1)
        Ks = odg.dg_operator(*sd, k, tuple(sd[d] * h[d] for d in range(3)), mask).tocsr()
        gidx = []
        for bz in range(sd[2]):
            for by in range(sd[1]):
                for bx in range(sd[0]):
                    gc = (lo[0] + bx) + dims[0] * ((lo[1] + by) + dims[1] * (lo[2] + bz))
                    gidx.append(gc * n3 + np.arange(n3))
        gidx = np.concatenate(gidx)
        xs = x[torch.tensor(gidx, device=DEV)].cpu().numpy()
        lc = (c[0] - lo[0]) + sd[0] * ((c[1] - lo[1]) + sd[1] * (c[2] - lo[2]))
        rows = lc * n3 + np.arange(n3)
        ref = Ks[rows] @ xs
        gc = c[0] + dims[0] * (c[1] + dims[1] * c[2])
        got = y[gc * n3:(gc + 1) * n3].cpu().numpy()
        got32 = y32[gc * n3:(gc + 1) * n3].cpu().double().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-12 * scale, (c, np.abs(got - ref).max() / scale)
        assert np.abs(got32 - ref).max() <= 1e-5 * scale, (c, np.abs(got32 - ref).max() / scale)


@pytest.mark.parametrize("mixed", [True, False])
def test_sipg_problems_in_a_batch_equal_their_standalone_solves(mfx, mixed):
    """SIPG operators share one batch with a continuous one: every result equals its own mfx_solve
    (both stop at a 1e-10 relative residual) and meets the residual bound of the oracle's matrix."""
    probs = []
    for dims, k in (((3, 2, 2), 2), ((2, 2, 2), 3)):
        op = sipg(mfx, dims, k)
        probs.append((op, odg.dg_operator(*dims, k), None))
    verts = synthetic.deformed_vertices(4, 4, 4)
    cg = mfx.Operator(mfx.Mesh.structured_box(4, 4, 4, verts), 2, mfx.COEF_TRIG, (1.0, 0.5))
    from oracle import mesh as omesh
    om = omesh.structured_mesh(4, 4, 4, 2, verts)
    probs.append((cg, fem.assemble(om, 3, fem.COEF_TRIG, (1.0, 0.5)), om))
    bs, alone = [], []
    for i, (op, K, om) in enumerate(probs):
        b = synthetic.uniform_vector(op.n_dofs, 80 + i)
        if om is not None:
            b[om.constrained] = 0.0
        bd = torch.tensor(b, device=DEV)
        x = torch.zeros_like(bd)
        st = op.solve(bd, x, tol=1e-10, mixed=mixed)
        assert st["status"] == 0
        bs.append(bd)
        alone.append(x.cpu().numpy())
    batch = mfx.Batch(4, chunk=4)
    xs, slots = [], []
    for (op, K, om), bd in zip(probs, bs):
        x = torch.full_like(bd, float("nan"))
        slots.append(batch.add(op, bd, x, tol=1e-10, mixed=mixed))
        xs.append(x)
    assert batch.run() > 0
    for (op, K, om), slot, bd, x, xa in zip(probs, slots, bs, xs, alone):
        done, st = batch.poll(slot)
        assert done and st["status"] == 0, st
        xb = x.cpu().numpy()
        b = bd.cpu().numpy()
        assert np.linalg.norm(b - K @ xb) <= 1.0001e-10 * np.linalg.norm(b)
        assert np.linalg.norm(xb - xa) <= 1e-8 * np.linalg.norm(xa)
        batch.release(slot)
