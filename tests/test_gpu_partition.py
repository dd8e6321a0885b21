"""GPU tests of the partitioned operator (the distributed path of Sec. 2.6 / Sec. 3.7) on one GPU.

Two or three parts of one structured box live in one process: each part's operator is built from its
slab of the global vertex lattice, its vmult gives its cells' contributions, and the shared planes are
exchanged by device copies and added with mfx_halo_accumulate.  The assembled result must equal the
oracle's global operator (1e-12 FP64, 1e-5 FP32).  The partitioned Jacobi-PCG runs one host thread per
part (the threads meet in the exchange and allreduce callbacks; no kernel of one part waits for
another) and must reach the global solution.
"""
import threading

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from oracle import mesh as omesh
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


def make_parts(mfx, nx, ny, nz, k, n_parts, verts, mask, precisions=3):
    parts = []
    for p in range(n_parts):
        info = mfx.partition_box(nx, ny, nz, k, n_parts, p, dirichlet=mask)
        nv = (nx + 1) * (ny + 1) * (info.nz + 1)
        mesh = mfx.Mesh.structured_box(nx, ny, info.nz, verts[info.vertex0:info.vertex0 + nv], dirichlet=info.dirichlet)
        op = mfx.Operator(mesh, k, mfx.COEF_TRIG, (1.0, 0.5), precisions=precisions)
        assert op.n_dofs == info.n_dofs
        parts.append((info, op))
    return parts


def partitioned_vmult(mfx, parts, x, dtype):
    ys = []
    for info, op in parts:
        xs = torch.tensor(x[info.dof0:info.dof0 + info.n_dofs], device=DEV, dtype=dtype)
        y = torch.empty_like(xs)
        op.vmult(xs, y)
        ys.append(y)
    # exchange: each part adds the neighbour's partial plane (copies of the partial planes taken first)
    P = parts[0][0].plane
    lo = [y[:P].clone() for y in ys]
    hi = [y[-P:].clone() for y in ys]
    for p, (info, op) in enumerate(parts):
        if info.has_lo:
            mfx.halo_accumulate(op, 0, hi[p - 1], ys[p])
        if info.has_hi:
            mfx.halo_accumulate(op, 1, lo[p + 1], ys[p])
    torch.cuda.synchronize()
    out = np.zeros(len(x))
    for (info, _), y in zip(parts, ys):
        out[info.dof0:info.dof0 + info.n_dofs] = y.double().cpu().numpy()
    return out, ys


@pytest.mark.parametrize("n_parts,k,mask", [(2, 2, 0x3F), (3, 3, 0b011101), (2, 4, 0b101111)])
def test_partitioned_vmult_equals_the_global_operator(mfx, n_parts, k, mask):
    nx, ny, nz = 4, 3, 5
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts, dirichlet=mask)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    x = synthetic.uniform_vector(om.n_dofs, 60 + k)
    ref = K @ x
    parts = make_parts(mfx, nx, ny, nz, k, n_parts, verts, mask)
    y, ys = partitioned_vmult(mfx, parts, x, torch.float64)
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() < 1e-12 * scale
    # both copies of every shared plane agree (each part holds the global rows of its whole slice)
    P = parts[0][0].plane
    for p in range(n_parts - 1):
        assert torch.equal(ys[p][-P:], ys[p + 1][:P])
    y32, _ = partitioned_vmult(mfx, parts, x, torch.float32)
    assert np.linalg.norm(y32 - ref) < 1e-5 * np.linalg.norm(ref)


def test_partitioned_solve_two_threads(mfx):
    nx, ny, nz, k, n_parts = 4, 3, 6, 3, 2
    verts = synthetic.deformed_vertices(nx, ny, nz)
    om = omesh.structured_mesh(nx, ny, nz, k, verts)
    K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
    b = synthetic.gaussian_vector(om.n_dofs, 9)
    b[om.constrained] = 0.0
    parts = make_parts(mfx, nx, ny, nz, k, n_parts, verts, 0x3F)
    P = parts[0][0].plane
    send = [[torch.empty(P, dtype=torch.float64, device=DEV) if s else None
             for s in (info.has_lo, info.has_hi)] for info, _ in parts]
    recv = [[torch.empty(P, dtype=torch.float64, device=DEV) if s else None
             for s in (info.has_lo, info.has_hi)] for info, _ in parts]
    bar = threading.Barrier(n_parts, timeout=120)
    sums = {}
    results = [None] * n_parts
    errors = []

    def run(p):
        try:
            info, op = parts[p]
            torch.cuda.set_device(0)

            def exchange():
                bar.wait()  # every part's send planes are ready
                if info.has_lo:
                    recv[p][0].copy_(send[p - 1][1])
                if info.has_hi:
                    recv[p][1].copy_(send[p + 1][0])
                torch.cuda.synchronize()
                bar.wait()  # nobody overwrites a send plane before the neighbour has copied it

            def allreduce(vals):
                sums[p] = np.asarray(vals)
                bar.wait()
                total = sum(sums[q] for q in range(n_parts))
                bar.wait()
                return total

            bd = torch.tensor(b[info.dof0:info.dof0 + info.n_dofs], device=DEV)
            xd = torch.zeros_like(bd)
            st = mfx.solve_partitioned(op, info, bd, xd, exchange, allreduce, send[p], recv[p], tol=1e-10)
            results[p] = (st, xd.cpu().numpy())
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)
            bar.abort()

    threads = [threading.Thread(target=run, args=(p,)) for p in range(n_parts)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    x = np.zeros(om.n_dofs)
    for (info, _), (st, xp) in zip(parts, results):
        assert st["status"] == 0 and st["rel_residual"] <= 1.0001e-10, st
        x[info.dof0:info.dof0 + info.n_dofs] = xp
    assert results[0][0]["iterations"] == results[1][0]["iterations"]
    assert np.linalg.norm(b - K @ x) <= 1.001e-10 * np.linalg.norm(b)
    xs = spla.spsolve(K.tocsc(), b)
    assert np.linalg.norm(x - xs) < 1e-8 * np.linalg.norm(xs)
    # the same iterations as the single-operator Jacobi-PCG, within one
    op = mfx.Operator(mfx.Mesh.structured_box(nx, ny, nz, verts), k, mfx.COEF_TRIG, (1.0, 0.5))
    xg = torch.zeros(om.n_dofs, dtype=torch.float64, device=DEV)
    stg = op.solve(torch.tensor(b, device=DEV), xg, tol=1e-10)
    assert abs(stg["iterations"] - results[0][0]["iterations"]) <= 1
