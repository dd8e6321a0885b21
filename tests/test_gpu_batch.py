"""Batched solves: every problem's result is the same alone (mfx_solve) and in the mix (mfx_batch).

Problems of different degree, size and mesh kind (structured, octree with hanging nodes) share one batch;
each result must match its own stand-alone solve within 1e-9 relative (both stop at a 1e-10 relative
residual) and satisfy the residual bound against the oracle's assembled matrix.
"""
import numpy as np
import pytest

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


def problems(mfx):
    out = []
    for i, (nx, k) in enumerate([(4, 1), (5, 2), (3, 3), (6, 1), (2, 4)]):
        verts = synthetic.deformed_vertices(nx, nx, nx)
        op = mfx.Operator(mfx.Mesh.structured_box(nx, nx, nx, verts), k, mfx.COEF_TRIG, (1.0, 0.5))
        om = omesh.structured_mesh(nx, nx, nx, k, verts)
        out.append((op, om))
    leaves = synthetic.octree_leaves(3, 1, (0.5, 0.5, 0.5), 0.3)
    op = mfx.Operator(mfx.Mesh.octree(3, 3, 3, leaves), 2)
    out.append((op, omesh.octree_mesh(3, 3, 3, 2, leaves)))
    return out


@pytest.mark.parametrize("mixed", [True, False])
def test_batch_results_equal_standalone_results(mfx, mixed):
    probs = problems(mfx)
    bs, alone, kmats = [], [], []
    for i, (op, om) in enumerate(probs):
        b = synthetic.uniform_vector(op.n_dofs, 60 + i)
        b[om.constrained] = 0.0
        bd = torch.tensor(b, device="cuda")
        x = torch.zeros_like(bd)
        st = op.solve(bd, x, tol=1e-10, mixed=mixed)
        assert st["status"] == 0
        bs.append(bd)
        alone.append(x.cpu().numpy())
    batch = mfx.Batch(8, chunk=4)
    xs, slots = [], []
    for (op, om), bd in zip(probs, bs):
        x = torch.full_like(bd, float("nan"))
        slots.append(batch.add(op, bd, x, tol=1e-10, mixed=mixed))
        xs.append(x)
    ticks = batch.run()
    assert ticks > 0
    for i, ((op, om), slot) in enumerate(zip(probs, slots)):
        done, st = batch.poll(slot)
        assert done and st["status"] == 0, st
        xb = xs[i].cpu().numpy()
        assert np.linalg.norm(xb - alone[i]) <= 1e-9 * np.linalg.norm(alone[i])
        K = fem.assemble(om, om.k + 1, fem.COEF_TRIG if i < 5 else fem.COEF_CONSTANT,
                         (1.0, 0.5) if i < 5 else (1.0, 0.0))
        b = bs[i].cpu().numpy()
        assert np.linalg.norm(b - K @ xb) <= 1.0001e-10 * np.linalg.norm(b)
        batch.release(slot)


def test_batch_slot_reuse_and_busy_operator(mfx):
    op = mfx.Operator(mfx.Mesh.structured_box(4, 4, 4), 2)
    b = torch.tensor(synthetic.uniform_vector(op.n_dofs, 70), device="cuda")
    op.distribute(b)
    x = torch.zeros_like(b)
    batch = mfx.Batch(2)
    s = batch.add(op, b, x, mixed=True)
    with pytest.raises(mfx.MfxError) as e:
        batch.add(op, b, x)
    assert e.value.code == mfx.EBUSY
    batch.run()
    batch.release(s)
    x2 = torch.zeros_like(b)
    s2 = batch.add(op, b, x2, mixed=True)
    batch.run()
    assert batch.poll(s2)[0]
    assert torch.allclose(x, x2, rtol=0, atol=1e-12 * x.abs().max().item())
