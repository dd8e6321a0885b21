"""GPU parity of every FP32 vmult kernel of structured meshes against the FP64 oracle.

The structured FP32 vmult has several kernels (ten-phase collocation form, five-phase form with the
metric read at its point of use or staged in shared memory) and two compiled batch sizes per degree;
the autotuner picks one pair per mesh.  Each is compared here, element by element, with the oracle's
assembled condensed matrix (full quadrature, Sec. 2.4 / Sec. 3.6) on meshes whose rows of cells hold
at least two full batches and a ragged tail, on degenerate rows of one and two cells, and with
natural (non-Dirichlet) faces.  FP32 tolerance: 1e-5 relative, norm-wise and per entry against the
max-norm (single-precision sums of O(100) terms give about 1e-6).
"""
import numpy as np
import pytest

from oracle import fem
from oracle import mesh as omesh
from paper_1910_13247_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
TOL32 = 1e-5
# compiled batch sizes (cells per batch) per degree
BATCH_SIZES = {1: (32,), 2: (16, 32), 3: (16, 8), 4: (16, 8)}


@pytest.fixture(scope="module")
def mfx():
    from paper_1910_13247_gb300 import build, mfx as m
    build.build()
    m.lib()
    return m


def kernels(mfx):
    return (mfx.KERNEL_TEN_PHASE, mfx.KERNEL_FIVE_PHASE, mfx.KERNEL_FIVE_PHASE_STAGED)


def vmult(op, x, dtype):
    xd = torch.tensor(x, device=DEV, dtype=dtype)
    yd = torch.empty_like(xd)
    op.vmult(xd, yd)
    torch.cuda.synchronize()
    op.device_check()
    return yd.double().cpu().numpy()


def errs(y, ref):
    return np.linalg.norm(y - ref) / np.linalg.norm(ref), np.abs(y - ref).max() / np.abs(ref).max()


def oracle_case(nx, ny, nz, k, seed, dirichlet=0x3F):
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts, dirichlet=dirichlet)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, seed)
    return verts, om, K, x


def make_op(mfx, nx, ny, nz, k, verts, cb, kern, dirichlet=0x3F):
    m = mfx.Mesh.structured_box(nx, ny, nz, verts, dirichlet=dirichlet)
    op = mfx.Operator(m, k, mfx.COEF_TRIG, (1.0, 0.5), cells_per_block=cb, structured_kernel=kern)
    info = op.info()
    assert info["cells_per_block"] == cb and info["structured_kernel"] == kern
    return op


@pytest.mark.parametrize("k", sorted(BATCH_SIZES))
def test_full_batches_and_ragged_tail_every_kernel(mfx, k):
    """Rows of 2 CB + 3 cells (two full batches and a 3-cell tail) for every compiled batch size and
    every FP32 kernel; the FP64 vmult of the same operator is checked at 1e-12."""
    for cb in BATCH_SIZES[k]:
        nx, ny, nz = 2 * cb + 3, 2, 2
        verts, om, K, x = oracle_case(nx, ny, nz, k, 500 + 10 * k + cb)
        ref = K @ x
        for kern in kernels(mfx):
            op = make_op(mfx, nx, ny, nz, k, verts, cb, kern)
            e2, einf = errs(vmult(op, x, torch.float32), ref)
            assert e2 < TOL32 and einf < TOL32, (cb, kern, e2, einf)
        e2, einf = errs(vmult(op, x, torch.float64), ref)
        assert e2 < 1e-12 and einf < 1e-12, (cb, e2, einf)


@pytest.mark.parametrize("k", sorted(BATCH_SIZES))
@pytest.mark.parametrize("dims", [(1, 3, 2), (2, 2, 3), (5, 1, 1)])
def test_degenerate_rows_every_kernel(mfx, k, dims):
    """Rows of one, two and five cells: a single partial batch, pairs whose second cell is absent."""
    verts, om, K, x = oracle_case(*dims, k, 600 + k)
    ref = K @ x
    for kern in kernels(mfx):
        op = make_op(mfx, *dims, k, verts, BATCH_SIZES[k][0], kern)
        e2, einf = errs(vmult(op, x, torch.float32), ref)
        assert e2 < TOL32 and einf < TOL32, (dims, kern, e2, einf)


@pytest.mark.parametrize("k", [2, 4])
@pytest.mark.parametrize("mask", [0b000001, 0b110100, 0])
def test_natural_faces_every_kernel(mfx, k, mask):
    """Dirichlet on a subset of the faces (x-low only; y-low and both z faces; none): the natural faces'
    points are free rows and take the x-point merging and the output ownership of the kernels."""
    nx, ny, nz = 19, 3, 2
    verts, om, K, x = oracle_case(nx, ny, nz, k, 700 + k + mask, dirichlet=mask)
    ref = K @ x
    for cb in BATCH_SIZES[k]:
        for kern in kernels(mfx):
            op = make_op(mfx, nx, ny, nz, k, verts, cb, kern, dirichlet=mask)
            e2, einf = errs(vmult(op, x, torch.float32), ref)
            assert e2 < TOL32 and einf < TOL32, (cb, kern, mask, e2, einf)


def test_autotuned_choice_is_a_compiled_pair(mfx):
    """The autotuner (no request) picks one of the compiled (batch size, kernel) pairs, and its result
    equals the oracle's."""
    k, (nx, ny, nz) = 4, (35, 3, 2)
    verts, om, K, x = oracle_case(nx, ny, nz, k, 800)
    op = mfx.Operator(mfx.Mesh.structured_box(nx, ny, nz, verts), k, mfx.COEF_TRIG, (1.0, 0.5))
    info = op.info()
    assert info["cells_per_block"] in BATCH_SIZES[k]
    assert info["structured_kernel"] in kernels(mfx)
    e2, einf = errs(vmult(op, x, torch.float32), K @ x)
    assert e2 < TOL32 and einf < TOL32


@pytest.mark.parametrize("k,cb,dims", [(4, 8, d) for d in ((1, 1, 1), (5, 1, 1), (9, 2, 1), (12, 1, 2))] +
                         [(3, 16, d) for d in ((1, 1, 1), (4, 2, 2), (2, 3, 2), (2, 2, 2), (17, 1, 1))])
def test_packed_rows_clipped_at_the_vector_end(mfx, k, cb, dims):
    """The staged kernel moves tile rows with untiled bulk copies where it packs them (Q4 with 8 cells per
    batch, Q3 with 16): the tile row that reaches past the end of the vector is clipped to whole 16-byte
    words and its last 0..3 points go through plain loads and atomics.  At Q4 that row always keeps one
    point beyond its words (lattice rows of 4 nx + 1 points); the Q3 cases give 0, 1, 2 and 3."""
    nx, ny, nz = dims
    Mx, My, Mz = k * nx + 1, k * ny + 1, k * nz + 1
    n = Mx * My * Mz
    x0 = k * ((nx - 1) // cb) * cb       # first lattice point of the last batch of the last row
    g0 = (n - Mx + x0) & ~3              # 16-byte aligned start of the last tile row
    assert n - g0 <= 4 * ((k * cb + 7) // 4)  # the row's box reaches past the vector's end
    verts, om, K, x = oracle_case(nx, ny, nz, k, 900 + nx + 10 * ny + 100 * nz)
    op = make_op(mfx, nx, ny, nz, k, verts, cb, mfx.KERNEL_FIVE_PHASE_STAGED)
    e2, einf = errs(vmult(op, x, torch.float32), K @ x)
    assert e2 < TOL32 and einf < TOL32, (dims, (n - g0) % 4, e2, einf)


def test_misaligned_vectors_rejected_before_launch(mfx):
    """The FP32 structured kernels move tile rows with the copy engine, which needs 16-byte aligned
    vectors: a view starting one float into an allocation is rejected with MFX_EINVAL on the host, before
    anything is launched, and the aligned call still works."""
    k, (nx, ny, nz) = 4, (9, 2, 2)
    verts, om, K, x = oracle_case(nx, ny, nz, k, 950)
    op = make_op(mfx, nx, ny, nz, k, verts, 8, mfx.KERNEL_FIVE_PHASE_STAGED)
    big = torch.zeros(op.n_dofs + 4, device=DEV, dtype=torch.float32)
    src = big[1:1 + op.n_dofs]
    src.copy_(torch.tensor(x, device=DEV, dtype=torch.float32))
    y = torch.empty(op.n_dofs, device=DEV, dtype=torch.float32)
    with pytest.raises(mfx.MfxError) as e:
        op.vmult(src, y)
    assert e.value.code == mfx.EINVAL
    e2, einf = errs(vmult(op, x, torch.float32), K @ x)
    assert e2 < TOL32 and einf < TOL32
