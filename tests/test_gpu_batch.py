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


@pytest.mark.parametrize("one_launch", [False, True])
@pytest.mark.parametrize("mixed", [True, False])
def test_batch_results_equal_standalone_results(mfx, mixed, one_launch):
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
    if one_launch:
        assert batch.run_once() == len(probs)
    else:
        assert batch.run() > 0
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


@pytest.mark.parametrize("mixed", [True, False])
@pytest.mark.parametrize("independent", [False, True, "one_launch"])
def test_batch_degenerate_right_hand_sides(mfx, mixed, independent):
    """A zero right-hand side finishes with x = 0 and status OK, a NaN one with MFX_BREAKDOWN, and a
    regular one beside them converges; both schedulers (ticks and independent stepping), both modes."""
    ops = [mfx.Operator(mfx.Mesh.structured_box(4, 4, 4), 2) for _ in range(3)]
    b0 = torch.tensor(synthetic.uniform_vector(ops[0].n_dofs, 71), device="cuda")
    ops[0].distribute(b0)
    bz = torch.zeros_like(b0)
    bn = b0.clone()
    bn[bn.numel() // 2] = float("nan")
    batch = mfx.Batch(4, chunk=4)
    xs = [torch.full_like(b0, float("nan")) for _ in range(3)]
    slots = [batch.add(op, b, x, tol=1e-10, mixed=mixed) for op, b, x in zip(ops, (b0, bz, bn), xs)]
    if independent == "one_launch":
        assert batch.run_once() == 3
    elif independent:
        for _ in range(200000):
            if batch.advance() == 0:
                break
    else:
        batch.run()
    st = [batch.poll(s) for s in slots]
    assert all(d for d, _ in st), st
    assert st[0][1]["status"] == 0 and st[0][1]["rel_residual"] <= 1.0001e-10
    assert st[1][1]["status"] == 0 and torch.count_nonzero(xs[1]).item() == 0
    assert st[2][1]["status"] == mfx.BREAKDOWN


def test_operator_release_after_batch_completion(mfx):
    """An operator whose slot reported done is freed in stream order (no device-wide wait); a new
    operator made afterwards reuses the memory and still gives the same solution."""
    def solve_once():
        op = mfx.Operator(mfx.Mesh.structured_box(5, 5, 5), 3).prepare_solver()
        b = torch.tensor(synthetic.uniform_vector(op.n_dofs, 72), device="cuda")
        op.distribute(b)
        x = torch.zeros_like(b)
        batch = mfx.Batch(1)
        s = batch.add(op, b, x, mixed=True)
        while batch.advance() > 0:
            pass
        done, st = batch.poll(s)
        assert done and st["status"] == 0
        batch.release(s)
        op.release()
        assert op.handle is None
        return x.cpu()
    x1 = solve_once()
    x2 = solve_once()
    # the FP32 inner solves scatter with reduce-adds whose order varies: equal up to rounding
    assert torch.allclose(x1, x2, rtol=0, atol=1e-12 * x1.abs().max().item())


@pytest.mark.parametrize("mixed", [True, False])
def test_one_launch_caps_end_every_loop(mfx, mixed):
    """A tolerance no solve can reach ends every device-decided loop at its cap: NOT_CONVERGED after
    max_it outer corrections (mixed) or max_it iterations (FP64), and the launch returns."""
    op = mfx.Operator(mfx.Mesh.structured_box(4, 4, 4), 2)
    b = torch.tensor(synthetic.uniform_vector(op.n_dofs, 73), device="cuda")
    op.distribute(b)
    x = torch.zeros_like(b)
    batch = mfx.Batch(2, chunk=4)
    s = batch.add(op, b, x, tol=0.0, mixed=mixed, max_it=3 if mixed else 10, inner_max_it=6)
    assert batch.run_once() == 1
    done, st = batch.poll(s)
    assert done and st["status"] == mfx.NOT_CONVERGED, st
    if mixed:
        assert st["iterations"] == 3 and st["inner_iterations"] <= 3 * 6
    else:
        assert st["iterations"] == 10


@pytest.mark.parametrize("mixed", [True, False])
def test_one_launch_with_chebyshev_preconditioner(mfx, mixed):
    """Chebyshev(5)-Jacobi-preconditioned solves in one launch (the preconditioner's kernels inside the
    device-decided loops) equal the same solves alone within 1e-9 and meet the residual bound."""
    probs = problems(mfx)[:4]
    batch = mfx.Batch(4, chunk=4)
    xs, alone, bs, slots = [], [], [], []
    for i, (op, om) in enumerate(probs):
        b = synthetic.uniform_vector(op.n_dofs, 80 + i)
        b[om.constrained] = 0.0
        bd = torch.tensor(b, device="cuda")
        xa = torch.zeros_like(bd)
        st = op.solve(bd, xa, tol=1e-10, mixed=mixed, precond=mfx.PRECOND_CHEBYSHEV, cheb_degree=5)
        assert st["status"] == 0
        alone.append(xa.cpu().numpy())
        x = torch.full_like(bd, float("nan"))
        slots.append(batch.add(op, bd, x, tol=1e-10, mixed=mixed, precond=mfx.PRECOND_CHEBYSHEV, cheb_degree=5))
        xs.append(x)
        bs.append(b)
    assert batch.run_once() == len(probs)
    for i, ((op, om), slot) in enumerate(zip(probs, slots)):
        done, st = batch.poll(slot)
        assert done and st["status"] == 0, st
        xb = xs[i].cpu().numpy()
        assert np.linalg.norm(xb - alone[i]) <= 1e-9 * np.linalg.norm(alone[i])
        K = fem.assemble(om, om.k + 1, fem.COEF_TRIG, (1.0, 0.5))
        assert np.linalg.norm(bs[i] - K @ xb) <= 1.0001e-10 * np.linalg.norm(bs[i])
