"""GPU parity of the CUDA path against the FP64 oracle (element by element).

Tolerances: FP64 vmult / diagonal / right-hand side within 1e-12 relative,
norm-wise and per entry against the max-norm; FP32 vmult within 1e-5
norm-wise (single-precision arithmetic with FP32 accumulation over
O(100) terms per entry gives about 1e-6).  Integer tables are bit-exact
(tested on the CPU in test_abi.py).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from oracle import mesh as omesh
from paper_1910_13247_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mfx():
    from paper_1910_13247_gb300 import build, mfx as m
    build.build()
    m.lib()
    return m


DEV = "cuda:0"


def rel_err(y, ref):
    return np.linalg.norm(y - ref) / np.linalg.norm(ref), np.abs(y - ref).max() / np.abs(ref).max()


def run_vmult(op, x, dtype):
    xd = torch.tensor(x, device=DEV, dtype=dtype)
    yd = torch.empty_like(xd)
    op.vmult(xd, yd)
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


def make_pair(mfx, nx, ny, nz, k, deformed=True, coef=1):
    verts = synthetic.deformed_vertices(nx, ny, nz) if deformed else None
    m = mfx.Mesh.structured_box(nx, ny, nz, verts)
    par = (1.0, 0.5) if coef == 1 else (1.0, 0.0)
    op = mfx.Operator(m, k, coef, par)
    om = omesh.structured_mesh(nx, ny, nz, k, verts)
    return op, om, par


def test_config1_cartesian_q2_vmult(mfx):
    op, om, par = make_pair(mfx, 8, 8, 8, 2, deformed=False, coef=0)
    assert op.n_dofs == 4913
    K = fem.assemble(om, 3)
    x = synthetic.uniform_vector(om.n_dofs, 1)
    ref = K @ x
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12
    e32, _ = rel_err(run_vmult(op, x, torch.float32), ref)
    assert e32 < 1e-5


SIZES = {1: (7, 5, 6), 2: (6, 6, 6), 3: (5, 4, 3), 4: (4, 4, 4), 5: (3, 3, 3), 6: (3, 2, 2), 7: (2, 2, 2), 8: (2, 2, 1)}


@pytest.mark.parametrize("k", sorted(SIZES))
def test_deformed_variable_coefficient_vmult_all_degrees(mfx, k):
    op, om, par = make_pair(mfx, *SIZES[k], k)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, par)
    x = synthetic.uniform_vector(om.n_dofs, 10 + k)
    ref = K @ x
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    e32, _ = rel_err(run_vmult(op, x, torch.float32), ref)
    assert e32 < 1e-5, e32
    # diagonal
    d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.diagonal(d)
    dref = fem.diagonal(K)
    assert np.abs(d.cpu().numpy() - dref).max() < 1e-12 * np.abs(dref).max()


BATCH_SIZES = {2: (16, 32), 3: (16, 8), 4: (16, 8)}


@pytest.mark.parametrize("k", sorted(BATCH_SIZES))
def test_both_batch_sizes_and_autotuned_choice(mfx, k):
    """Structured kernels compiled for two batch sizes (metric laid out per choice) give the oracle's
    result on rows that are not a multiple of either; the autotuner picks one of them."""
    nx, ny, nz = 13, 3, 2
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, 90 + k)
    ref = K @ x
    for cb in BATCH_SIZES[k] + (0,):
        op = mfx.Operator(mfx.Mesh.structured_box(nx, ny, nz, verts), k, mfx.COEF_TRIG, (1.0, 0.5),
                          cells_per_block=cb)
        assert op.info()["cells_per_block"] in BATCH_SIZES[k]
        if cb:
            assert op.info()["cells_per_block"] == cb
        e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
        assert e2 < 1e-12 and einf < 1e-12, (cb, e2, einf)
        assert rel_err(run_vmult(op, x, torch.float32), ref)[0] < 1e-5
        d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
        op.diagonal(d)
        dref = fem.diagonal(K)
        assert np.abs(d.cpu().numpy() - dref).max() < 1e-12 * np.abs(dref).max(), cb


def test_quadrature_points_and_rhs(mfx):
    op, om, par = make_pair(mfx, 3, 4, 2, 3)
    X, _ = fem.quadrature_points(om, 4)
    xq = torch.empty(op.n_cells * 64 * 3, dtype=torch.float64, device=DEV)
    op.quadrature_points(xq)
    assert np.abs(xq.cpu().numpy().reshape(X.shape) - X).max() < 1e-15
    fq = synthetic.uniform_vector(op.n_cells * 64, 7)
    b = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.rhs(torch.tensor(fq, device=DEV), b)
    bref = fem.rhs(om, 4, fq=fq.reshape(op.n_cells, 64))
    e2, einf = rel_err(b.cpu().numpy(), bref)
    assert e2 < 1e-12 and einf < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_octree_vmult_with_hanging_nodes(mfx, k):
    g = synthetic.rng(200 + k)
    leaves = synthetic.octree_leaves(3, 2, g.uniform(0.3, 0.7, 3), 0.3)
    verts = synthetic.deformed_vertices(3, 3, 3)
    m = mfx.Mesh.octree(3, 3, 3, leaves, verts)
    op = mfx.Operator(m, k, mfx.COEF_TRIG, (1.0, 0.5))
    om = omesh.octree_mesh(3, 3, 3, k, leaves, verts)
    assert op.info()["n_hanging"] > 0
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, 20 + k)
    ref = K @ x
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    e32, _ = rel_err(run_vmult(op, x, torch.float32), ref)
    assert e32 < 1e-5
    d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.diagonal(d)
    dref = fem.diagonal(K)
    assert np.abs(d.cpu().numpy() - dref).max() < 1e-12 * np.abs(dref).max()
    # distribute fills hanging values from their masters
    xs = torch.tensor(x, device=DEV)
    op.distribute(xs)
    assert np.abs(xs.cpu().numpy() - fem.distribute(om, x)).max() < 1e-14


@pytest.mark.parametrize("seed,k,nb,radius", [(1, 3, 3, 0.25), (5, 4, 3, 0.25), (2, 5, 2, 0.25), (3, 6, 2, 0.35)])
def test_octree_tensor_product_hanging_constraints(mfx, seed, k, nb, radius):
    """Octrees refined twice around a seeded centre, at the degrees whose vmult applies the hanging
    constraints in tensor-product form (faces, and edges hanging on their own at the rim of the
    refined region): vmult equals the oracle's condensed matrix."""
    g = synthetic.rng(300 + seed)
    leaves = synthetic.octree_leaves(nb, 2, g.uniform(0.3, 0.7, 3), radius)
    verts = synthetic.deformed_vertices(nb, nb, nb)
    m = mfx.Mesh.octree(nb, nb, nb, leaves, verts)
    op = mfx.Operator(m, k, mfx.COEF_TRIG, (1.0, 0.5))
    assert op.info()["n_hanging"] > 0
    om = omesh.octree_mesh(nb, nb, nb, k, leaves, verts)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, 40 + seed)
    ref = K @ x
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    e32, _ = rel_err(run_vmult(op, x, torch.float32), ref)
    assert e32 < 1e-5, e32


@pytest.mark.parametrize("k,nb,levels,radius", [(1, 4, 2, 0.3), (2, 3, 2, 0.3), (3, 3, 1, 0.3), (4, 3, 2, 0.25),
                                              (6, 2, 1, 0.2), (7, 2, 1, 0.2), (8, 2, 1, 0.2), (8, 2, 1, 0.0)])
def test_octree_box_cell_metric(mfx, k, nb, levels, radius, monkeypatch):
    """Octree on the undeformed lattice with a constant coefficient: every cell is an axis-aligned box,
    and the FP32 kernels take the metric as one diagonal per cell (the paired kernel at k = 1 and at k = 8
    without hanging nodes, the five-phase kernel with and without hanging cells elsewhere; k = 7 keeps the
    full metric). FP32 and FP64 against the oracle, and the FP32 result against the same operator with
    the full metric (MFX_BOX_METRIC=0); a deformed lattice or a variable coefficient keeps the full metric."""
    g = synthetic.rng(500 + k)
    center = np.array([0.3, 0.3, 0.3]) if nb == 2 else g.uniform(0.3, 0.7, 3)
    leaves = synthetic.octree_leaves(nb, levels, center, radius)
    op = mfx.Operator(mfx.Mesh.octree(nb, nb, nb, leaves), k)
    info = op.info()
    assert (info["n_hanging"] > 0) == (radius > 0)
    assert info["box_metric"] == (0 if k == 7 else 1)
    om = omesh.octree_mesh(nb, nb, nb, k, leaves)
    K = fem.assemble(om, k + 1)
    x = synthetic.uniform_vector(om.n_dofs, 60 + k)
    ref = K @ x
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    y32 = run_vmult(op, x, torch.float32)
    e32, e32inf = rel_err(y32, ref)
    assert e32 < 1e-5 and e32inf < 1e-5, (e32, e32inf)
    monkeypatch.setenv("MFX_BOX_METRIC", "0")
    full = mfx.Operator(mfx.Mesh.octree(nb, nb, nb, leaves), k)
    assert full.info()["box_metric"] == 0
    if k != 7:
        assert info["bytes_device"] < full.info()["bytes_device"]
    assert rel_err(run_vmult(full, x, torch.float32), y32)[0] < 1e-6
    monkeypatch.delenv("MFX_BOX_METRIC")
    deformed = mfx.Operator(mfx.Mesh.octree(nb, nb, nb, leaves, synthetic.deformed_vertices(nb, nb, nb)), k)
    assert deformed.info()["box_metric"] == 0
    variable = mfx.Operator(mfx.Mesh.octree(nb, nb, nb, leaves), k, mfx.COEF_TRIG, (1.0, 0.5))
    assert variable.info()["box_metric"] == 0


@pytest.mark.parametrize("k,kernel", [(1, "TEN_PHASE"), (2, "TEN_PHASE"), (3, "TEN_PHASE"), (4, "TEN_PHASE"),
                                      (5, "TEN_PHASE"), (1, "FIVE_PHASE"), (2, "FIVE_PHASE_STAGED"),
                                      (3, "FIVE_PHASE"), (4, "FIVE_PHASE_STAGED"), (4, "FIVE_PHASE")])
def test_structured_box_cell_metric_row_batch(mfx, k, kernel, monkeypatch):
    """Structured row-batch kernels on box cells with a constant coefficient read three entries of each
    line's FP32 metric (its first point's diagonal) and scale them by the quadrature weights: rows of 35
    cells (full and partial batches), FP32 against the oracle and against the full metric."""
    dims = (35, 3, 2)
    kid = getattr(mfx, "KERNEL_" + kernel)
    op = mfx.Operator(mfx.Mesh.structured_box(*dims), k, structured_kernel=kid)
    assert op.info()["box_metric"] == 1 and op.info()["structured_kernel"] == kid
    om = omesh.structured_mesh(*dims, k)
    K = fem.assemble(om, k + 1)
    x = synthetic.uniform_vector(om.n_dofs, 90 + k)
    ref = K @ x
    y32 = run_vmult(op, x, torch.float32)
    e2, einf = rel_err(y32, ref)
    assert e2 < 1e-5 and einf < 1e-5, (e2, einf)
    monkeypatch.setenv("MFX_BOX_METRIC", "0")
    full = mfx.Operator(mfx.Mesh.structured_box(*dims), k, structured_kernel=kid)
    assert full.info()["box_metric"] == 0
    assert rel_err(run_vmult(full, x, torch.float32), y32)[0] < 1e-6


@pytest.mark.parametrize("k,n", [(6, 3), (8, 2), (7, 2)])
def test_structured_box_cell_metric_high_degree(mfx, k, n, monkeypatch):
    """Structured meshes from k = 6 on run the per-cell kernels; on the undeformed cube with a constant
    coefficient their FP32 metric is one diagonal per cell too (not at k = 7): FP32 against the oracle and
    against the full metric."""
    op = mfx.Operator(mfx.Mesh.structured_box(n, n, n), k)
    assert op.info()["box_metric"] == (0 if k == 7 else 1)
    om = omesh.structured_mesh(n, n, n, k)
    K = fem.assemble(om, k + 1)
    x = synthetic.uniform_vector(om.n_dofs, 80 + k)
    ref = K @ x
    y32 = run_vmult(op, x, torch.float32)
    e2, einf = rel_err(y32, ref)
    assert e2 < 1e-5 and einf < 1e-5, (e2, einf)
    assert rel_err(run_vmult(op, x, torch.float64), ref)[0] < 1e-12
    monkeypatch.setenv("MFX_BOX_METRIC", "0")
    full = mfx.Operator(mfx.Mesh.structured_box(n, n, n), k)
    assert full.info()["box_metric"] == 0
    assert rel_err(run_vmult(full, x, torch.float32), y32)[0] < 1e-6


@pytest.mark.parametrize("k", [5, 7, 8])
def test_octree_diagonal_high_degree(mfx, k):
    """Diagonal and vmult on an octree at high degree: the diagonal's sum-factorised paths (cells with
    and without hanging nodes) and the FP32 octree kernels (five phases at k = 5 and 8, ten phases at
    k = 7)."""
    leaves = synthetic.octree_leaves(2, 1, np.array([0.3, 0.3, 0.3]), 0.2)
    verts = synthetic.deformed_vertices(2, 2, 2)
    m = mfx.Mesh.octree(2, 2, 2, leaves, verts)
    op = mfx.Operator(m, k, mfx.COEF_TRIG, (1.0, 0.5))
    om = omesh.octree_mesh(2, 2, 2, k, leaves, verts)
    assert op.info()["n_hanging"] > 0
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.diagonal(d)
    dref = fem.diagonal(K)
    assert np.abs(d.cpu().numpy() - dref).max() < 1e-12 * np.abs(dref).max()
    # vmult at high degree
    x = synthetic.uniform_vector(om.n_dofs, 40 + k)
    ref = K @ x
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    assert rel_err(run_vmult(op, x, torch.float32), ref)[0] < 1e-5


def test_single_cell_degenerate_meshes(mfx):
    # one Q1 cell: every DoF is on the boundary, the operator is the identity
    m = mfx.Mesh.structured_box(1, 1, 1)
    op = mfx.Operator(m, 1)
    x = synthetic.uniform_vector(8, 3)
    assert np.array_equal(run_vmult(op, x, torch.float64), x)
    # one Q8 cell: a single cell with 729 nodes, 343 of them free
    op, om, par = make_pair(mfx, 1, 1, 1, 8)
    K = fem.assemble(om, 9, fem.COEF_TRIG, par)
    x = synthetic.uniform_vector(om.n_dofs, 4)
    e2, _ = rel_err(run_vmult(op, x, torch.float64), K @ x)
    assert e2 < 1e-12


@pytest.mark.parametrize("nx,k", [(64, 4), (96, 3)])
def test_full_size_sampled_rows(mfx, nx, k):
    """Full-size workloads (64^3 Q4 and 96^3 Q3, deformed, variable coefficient) in the benchmark's
    launch configuration: sampled rows against the oracle's row-by-row product."""
    verts = synthetic.deformed_vertices(nx, nx, nx)
    m = mfx.Mesh.structured_box(nx, nx, nx, verts)
    op = mfx.Operator(m, k, mfx.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(op.n_dofs, 2)
    y = run_vmult(op, x, torch.float64)
    y32 = run_vmult(op, x, torch.float32)
    # the oracle's sampled rows need only the cells of each DoF: build them from a sub-mesh view
    rows = synthetic.rng(5).choice(op.n_dofs, 300, replace=False)
    ref = sampled_rows_structured(nx, k, verts, x, rows)
    scale = np.abs(ref).max()
    assert np.abs(y[rows] - ref).max() < 1e-12 * scale
    # FP32, in the launch configuration the autotuner chose (the benchmark's), against the oracle's rows
    assert np.abs(y32[rows] - ref).max() < 1e-5 * scale, op.info()
    assert np.linalg.norm(y32[rows] - ref) < 1e-5 * np.linalg.norm(ref)
    # and every other structured FP32 kernel at the autotuned batch size
    cb = op.info()["cells_per_block"]
    del op
    for kern in (mfx.KERNEL_TEN_PHASE, mfx.KERNEL_FIVE_PHASE, mfx.KERNEL_FIVE_PHASE_STAGED):
        opk = mfx.Operator(m, k, mfx.COEF_TRIG, (1.0, 0.5), precisions=2, cells_per_block=cb, structured_kernel=kern)
        y32k = run_vmult(opk, x, torch.float32)
        assert np.abs(y32k[rows] - ref).max() < 1e-5 * scale, kern
        del opk


def sampled_rows_structured(nx, k, verts, x, rows):
    """Oracle rows (K x)[rows] on the nx^3 structured mesh, from the element rows of each row's cells."""
    M = k * nx + 1
    out = np.zeros(len(rows))
    n = k + 1
    for t, d in enumerate(rows):
        I, J, L = d % M, (d // M) % M, d // (M * M)
        if min(I, J, L) == 0 or max(I, J, L) == M - 1:
            out[t] = x[d]
            continue
        s = 0.0
        for cz in {(L - 1) // k, L // k} & set(range(nx)):
            for cy in {(J - 1) // k, J // k} & set(range(nx)):
                for cx in {(I - 1) // k, I // k} & set(range(nx)):
                    i1, i2, i3 = I - k * cx, J - k * cy, L - k * cz
                    if not (0 <= i1 <= k and 0 <= i2 <= k and 0 <= i3 <= k):
                        continue
                    cell = omesh.structured_mesh(1, 1, 1, k, np.array(
                        [verts[(cx + a) + (nx + 1) * ((cy + b) + (nx + 1) * (cz + e))]
                         for e in (0, 1) for b in (0, 1) for a in (0, 1)]))
                    row = fem.element_matrices(cell, n, fem.COEF_TRIG, (1.0, 0.5), rows=[i1 + n * (i2 + n * i3)])[0, 0]
                    gd = np.array([(k * cx + a1) + M * ((k * cy + a2) + M * (k * cz + a3))
                                   for a3 in range(n) for a2 in range(n) for a1 in range(n)])
                    gI, gJ, gL = gd % M, (gd // M) % M, gd // (M * M)
                    bnd = (np.minimum(np.minimum(gI, gJ), gL) == 0) | (np.maximum(np.maximum(gI, gJ), gL) == M - 1)
                    s += float(row @ np.where(bnd, 0.0, x[gd]))
        out[t] = s
    return out


def test_dot_and_chebyshev(mfx):
    op, om, par = make_pair(mfx, 4, 4, 4, 3)
    K = fem.assemble(om, 4, fem.COEF_TRIG, par)
    a = synthetic.uniform_vector(om.n_dofs, 30)
    b = synthetic.uniform_vector(om.n_dofs, 31)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    op.dot(torch.tensor(a, device=DEV), torch.tensor(b, device=DEV), out)
    assert abs(out.item() - a @ b) < 1e-12 * np.abs(a) @ np.abs(b)
    d = fem.diagonal(K)
    lo, hi = 0.1, 2.5
    r = synthetic.uniform_vector(om.n_dofs, 32)
    zref = fem.chebyshev(lambda v: K @ v, 1 / d, r, 5, lo, hi)
    z = torch.empty(om.n_dofs, dtype=torch.float64, device=DEV)
    op.chebyshev(torch.tensor(r, device=DEV), z, 5, lo, hi)
    e2, einf = rel_err(z.cpu().numpy(), zref)
    assert e2 < 1e-12 and einf < 1e-12
    z32 = torch.empty(om.n_dofs, dtype=torch.float32, device=DEV)
    op.chebyshev(torch.tensor(r, device=DEV, dtype=torch.float32), z32, 5, lo, hi)
    assert rel_err(z32.double().cpu().numpy(), zref)[0] < 1e-5


def test_config1_jacobi_pcg_solve(mfx):
    op, om, par = make_pair(mfx, 8, 8, 8, 2, deformed=False, coef=0)
    K = fem.assemble(om, 3)
    b = fem.rhs(om, 3)
    bd = torch.tensor(b, device=DEV)
    x = torch.zeros_like(bd)
    st = op.solve(bd, x, tol=1e-10)
    assert st["status"] == 0, st
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - K @ xs) <= 1.0001e-10 * np.linalg.norm(b)
    ref = fem.pcg(lambda v: K @ v, b, lambda r: r / fem.diagonal(K), tol=1e-10)
    assert abs(st["iterations"] - ref.iterations) <= 1
    xd = spla.spsolve(K.tocsc(), b)
    assert np.linalg.norm(xs - xd) < 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("mixed", [False, True])
def test_chebyshev_pcg_and_mixed_precision_solve(mfx, mixed):
    op, om, par = make_pair(mfx, 6, 6, 6, 3)
    K = fem.assemble(om, 4, fem.COEF_TRIG, par)
    b = synthetic.gaussian_vector(om.n_dofs, 3)
    b[om.constrained] = 0.0
    bd = torch.tensor(b, device=DEV)
    x = torch.zeros_like(bd)
    st = op.solve(bd, x, tol=1e-10, precond=mfx.PRECOND_CHEBYSHEV, cheb_degree=5, mixed=mixed, inner_tol=1e-4)
    assert st["status"] == 0, st
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - K @ xs) <= 1.0001e-10 * np.linalg.norm(b)
    xd = spla.spsolve(K.tocsc(), b)
    assert np.linalg.norm(xs - xd) < 1e-8 * np.linalg.norm(xd)
    # the eigenvalue estimate is close to the oracle's on the same start vector
    d = fem.diagonal(K)
    lam = fem.lanczos_lambda_max(lambda v: K @ v, 1 / d, b, 15)
    assert abs(st["lambda_max"] - lam) < 1e-3 * lam


def test_bounded_wait_runs_out_and_is_reported(mfx):
    """Failure detection without a fault: a kernel waits on an mbarrier at which nothing arrives, through
    the bounded wait of the TMA kernels; the wait runs out after about a second, the operator's error word
    is set, device_check raises ETIMEOUT once (the word is cleared), and the operator keeps working."""
    import time
    op, om, par = make_pair(mfx, 3, 3, 3, 2)
    op.device_check()
    t0 = time.perf_counter()
    op.selftest_bounded_wait()
    with pytest.raises(mfx.MfxError) as e:
        op.device_check()
    dt = time.perf_counter() - t0
    assert e.value.code == mfx.ETIMEOUT
    assert 0.2 < dt < 30, dt
    op.device_check()
    K = fem.assemble(om, 3, fem.COEF_TRIG, par)
    x = synthetic.uniform_vector(om.n_dofs, 9)
    e2, einf = rel_err(run_vmult(op, x, torch.float64), K @ x)
    assert e2 < 1e-12 and einf < 1e-12


def test_solver_statuses(mfx):
    op, om, par = make_pair(mfx, 4, 4, 4, 2)
    b = synthetic.uniform_vector(om.n_dofs, 9)
    b[om.constrained] = 0.0
    bd = torch.tensor(b, device=DEV)
    x = torch.zeros_like(bd)
    st = op.solve(bd, x, tol=1e-10, max_it=3)
    assert st["status"] == mfx.NOT_CONVERGED and st["iterations"] == 3
    bn = bd.clone()
    bn[om.n_dofs // 2] = float("nan")
    st = op.solve(bn, x, tol=1e-10)
    assert st["status"] == mfx.BREAKDOWN
    z = torch.zeros_like(bd)
    st = op.solve(z, x, tol=1e-10)
    assert st["status"] == 0 and torch.count_nonzero(x).item() == 0


def test_mesh_transform_coefficient_and_rhs_functions(mfx):
    """Geometry by a host map of the vertices (mfx_mesh_transform), the coefficient as a host function
    (MFX_COEF_FUNCTION) and the load vector of a host function (mfx_rhs_function) give the operator and
    right-hand side of the same problem set up from vertex arrays and closed-form kinds."""
    import math

    def phi(x, y, z):
        d = 0.05 * math.sin(math.pi * x) * math.sin(math.pi * y) * math.sin(math.pi * z)
        return x + d, y + d, z + d

    def coef(x, y, z):
        return 1.0 + 0.5 * math.sin(2 * math.pi * x) * math.cos(2 * math.pi * y) * z

    nx, ny, nz, k = 4, 3, 3, 3
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, 33)
    ref = K @ x
    op = mfx.Operator(mfx.Mesh.structured_box(nx, ny, nz).transform(phi), k, coef_fn=coef)
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    # octree: the coarse lattice moves, leaves follow
    leaves = synthetic.octree_leaves(3, 1, np.array([0.4, 0.5, 0.5]), 0.3)
    oo = omesh.octree_mesh(3, 3, 3, 2, leaves, synthetic.deformed_vertices(3, 3, 3))
    Ko = fem.assemble(oo, 3, fem.COEF_TRIG, (1.0, 0.5))
    xo = synthetic.uniform_vector(oo.n_dofs, 34)
    opo = mfx.Operator(mfx.Mesh.octree(3, 3, 3, leaves).transform(phi), 2, coef_fn=coef)
    e2, einf = rel_err(run_vmult(opo, xo, torch.float64), Ko @ xo)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)

    # load vector of f(x) = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) against the oracle's
    def f(x, y, z):
        return 3 * math.pi ** 2 * math.sin(math.pi * x) * math.sin(math.pi * y) * math.sin(math.pi * z)

    b = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.rhs_function(f, b)
    Xq, _ = fem.quadrature_points(om, k + 1)
    fq = np.array([f(*p) for p in Xq.reshape(-1, 3)]).reshape(op.n_cells, (k + 1) ** 3)
    e2, einf = rel_err(b.cpu().numpy(), fem.rhs(om, k + 1, fq=fq))
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)


@pytest.mark.parametrize("faces", [0, 0b000011, 0b110100, 0b011001])
def test_dirichlet_face_masks(mfx, faces):
    """Dirichlet on a subset of the faces (natural boundaries elsewhere): FP64 / FP32 vmult of both
    structured batch layouts and of an octree with hanging nodes, the diagonal and (with at least one
    Dirichlet face) a PCG solve, against the oracle's operator built with the same mask."""
    nx, ny, nz, k = 13, 3, 2, 3  # rows not a multiple of either batch size
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts, dirichlet=faces)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, 50)
    ref = K @ x
    dref = fem.diagonal(K)
    for cb in (8, 16):
        op = mfx.Operator(mfx.Mesh.structured_box(nx, ny, nz, verts, dirichlet=faces), k, mfx.COEF_TRIG, (1.0, 0.5),
                          cells_per_block=cb)
        assert op.info()["n_constrained"] == len(om.constrained)
        e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
        assert e2 < 1e-12 and einf < 1e-12, (cb, e2, einf)
        assert rel_err(run_vmult(op, x, torch.float32), ref)[0] < 1e-5
        d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
        op.diagonal(d)
        assert np.abs(d.cpu().numpy() - dref).max() < 1e-12 * np.abs(dref).max(), cb
    if faces:
        b = synthetic.uniform_vector(om.n_dofs, 51)
        b[om.constrained] = 0.0
        bd = torch.tensor(b, device=DEV)
        xs = torch.zeros_like(bd)
        st = op.solve(bd, xs, tol=1e-10)
        assert st["status"] == 0
        assert np.linalg.norm(b - K @ xs.cpu().numpy()) <= 1.0001e-10 * np.linalg.norm(b)
    # octree: the refined ball touches the x = 0 and y = 0 faces
    leaves = synthetic.octree_leaves(3, 1, np.array([0.15, 0.2, 0.5]), 0.3)
    ov = synthetic.deformed_vertices(3, 3, 3)
    oo = omesh.octree_mesh(3, 3, 3, 2, leaves, ov, dirichlet=faces)
    Ko = fem.assemble(oo, 3, fem.COEF_TRIG, (1.0, 0.5))
    xo = synthetic.uniform_vector(oo.n_dofs, 52)
    opo = mfx.Operator(mfx.Mesh.octree(3, 3, 3, leaves, ov, dirichlet=faces), 2, mfx.COEF_TRIG, (1.0, 0.5))
    e2, einf = rel_err(run_vmult(opo, xo, torch.float64), Ko @ xo)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    d = torch.empty(opo.n_dofs, dtype=torch.float64, device=DEV)
    opo.diagonal(d)
    assert np.abs(d.cpu().numpy() - fem.diagonal(Ko)).max() < 1e-12 * np.abs(fem.diagonal(Ko)).max()
    xs = torch.tensor(xo, device=DEV)
    opo.distribute(xs)
    assert np.abs(xs.cpu().numpy() - fem.distribute(oo, xo)).max() < 1e-14


@pytest.mark.parametrize("faces", [0, 0b110100])
@pytest.mark.parametrize("k", [6, 7])
def test_high_degree_structured_dirichlet_face_masks(mfx, faces, k):
    """From k = 6 on, the FP32 vmult of a structured mesh runs on the per-cell kernels with an index table
    of the lattice built on the device (Dirichlet points as constraint rows): with natural faces the
    boundary points there are free DoFs. FP64 / FP32 vmult and diagonal against the oracle."""
    nx, ny, nz = 3, 2, 2
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts, dirichlet=faces)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, 70 + k)
    ref = K @ x
    op = mfx.Operator(mfx.Mesh.structured_box(nx, ny, nz, verts, dirichlet=faces), k, mfx.COEF_TRIG, (1.0, 0.5))
    assert op.info()["n_constrained"] == len(om.constrained)
    e2, einf = rel_err(run_vmult(op, x, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    assert rel_err(run_vmult(op, x, torch.float32), ref)[0] < 1e-5
    d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.diagonal(d)
    dref = fem.diagonal(K)
    assert np.abs(d.cpu().numpy() - dref).max() < 1e-12 * np.abs(dref).max()


@pytest.mark.parametrize("faces", [0, 0b000011, 0b110100])
@pytest.mark.parametrize("k", [3, 4])
def test_octree_tensor_product_with_dirichlet_face_masks(mfx, faces, k):
    """Octrees refined twice in a ball that reaches the x = 0 and y = 0 faces, at the degrees whose vmult
    applies the hanging constraints in tensor-product form, with Dirichlet on all, some or none of the
    faces: hanging nodes on natural faces keep their boundary masters, those on Dirichlet faces lose
    them. FP64 / FP32 vmult, diagonal and distribute against the oracle built with the same mask."""
    leaves = synthetic.octree_leaves(3, 2, np.array([0.15, 0.2, 0.5]), 0.3)
    ov = synthetic.deformed_vertices(3, 3, 3)
    oo = omesh.octree_mesh(3, 3, 3, k, leaves, ov, dirichlet=faces)
    Ko = fem.assemble(oo, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    xo = synthetic.uniform_vector(oo.n_dofs, 60 + k)
    ref = Ko @ xo
    op = mfx.Operator(mfx.Mesh.octree(3, 3, 3, leaves, ov, dirichlet=faces), k, mfx.COEF_TRIG, (1.0, 0.5))
    assert op.info()["n_hanging"] > 0 and op.info()["n_constrained"] == len(oo.constrained)
    e2, einf = rel_err(run_vmult(op, xo, torch.float64), ref)
    assert e2 < 1e-12 and einf < 1e-12, (e2, einf)
    assert rel_err(run_vmult(op, xo, torch.float32), ref)[0] < 1e-5
    d = torch.empty(op.n_dofs, dtype=torch.float64, device=DEV)
    op.diagonal(d)
    dref = fem.diagonal(Ko)
    assert np.abs(d.cpu().numpy() - dref).max() < 1e-12 * np.abs(dref).max()
    xs = torch.tensor(xo, device=DEV)
    op.distribute(xs)
    assert np.abs(xs.cpu().numpy() - fem.distribute(oo, xo)).max() < 1e-14


@pytest.mark.parametrize("count", [1, 2, 5])
def test_vmult_on_host_vectors(mfx, count):
    """mfx_vmult_host: the pipelined host-buffer path gives, for every vector, the oracle's product
    (FP64 within 1e-12, FP32 within 1e-5), on a structured and an octree operator."""
    nx, ny, nz, k = 5, 4, 3, 3
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    op = mfx.Operator(mfx.Mesh.structured_box(nx, ny, nz, verts), k, mfx.COEF_TRIG, (1.0, 0.5))
    leaves = synthetic.octree_leaves(3, 1, np.array([0.5, 0.5, 0.5]), 0.3)
    oo = omesh.octree_mesh(3, 3, 3, 2, leaves)
    Ko = fem.assemble(oo, 3)
    opo = mfx.Operator(mfx.Mesh.octree(3, 3, 3, leaves), 2)
    for o, KK, n in ((op, K, om.n_dofs), (opo, Ko, oo.n_dofs)):
        xs = [synthetic.uniform_vector(n, 60 + i) for i in range(count)]
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            src = [torch.tensor(x, dtype=dt).pin_memory() for x in xs]
            dst = [torch.full((n,), float("nan"), dtype=dt).pin_memory() for _ in xs]
            o.vmult_host(src, dst)
            for x, y in zip(xs, dst):
                assert rel_err(y.double().numpy(), KK @ x)[0] < tol
