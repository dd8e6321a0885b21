"""Serving: the library's native solve server admits requests while others run (continuous batching);
each result equals the same problem solved alone within 1e-9 relative; admission follows the memory
budget and the policy; cancel and retire follow the request's state."""
import time

import numpy as np
import pytest

from paper_1910_13247_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mfx():
    from paper_1910_13247_gb300 import build, mfx as m
    build.build()
    m.lib()
    return m


def wait_all(srv, tickets, mfx, limit=120.0):
    t0 = time.perf_counter()
    infos = {}
    while len(infos) < len(tickets):
        assert time.perf_counter() - t0 < limit, "server did not finish"
        for t in tickets:
            if t not in infos:
                i = srv.poll(t)
                if i["state"] >= mfx.REQ_DONE:
                    infos[t] = i
        time.sleep(0.001)
    return infos


def test_served_results_equal_standalone_solves(mfx):
    from paper_1910_13247_gb300 import serve
    reqs = serve.make_requests(10, rate=400.0, seed=11, size_range=(1e3, 4e4))
    server = serve.Server(budget_bytes=8 << 30, max_slots=4, chunk=8, keep_results=True)
    summary = server.run(reqs)
    assert summary["completed"] == 10 and summary["statuses"] == [0]
    assert summary["max_concurrent"] >= 2   # requests overlapped on the device
    for req in reqs:
        mesh = mfx.Mesh.octree(req.nb, req.nb, req.nb, req.leaves)
        op = mfx.Operator(mesh, req.degree)
        b = torch.tensor(synthetic.gaussian_vector(op.n_dofs, req.seed), device="cuda")
        op.distribute(b)
        x = torch.zeros_like(b)
        st = op.solve(b, x, tol=1e-10, mixed=True)
        assert st["status"] == 0
        xa = x.cpu().numpy()
        assert np.linalg.norm(req.result - xa) <= 1e-9 * np.linalg.norm(xa), req.rid


def test_admission_respects_the_memory_budget(mfx):
    from paper_1910_13247_gb300 import serve
    reqs = serve.make_requests(6, rate=1000.0, seed=12, size_range=(2e3, 2e4))
    # a budget below any single request still admits one at a time (never more than one active)
    server = serve.Server(budget_bytes=1, max_slots=4, chunk=8)
    summary = server.run(reqs)
    assert summary["completed"] == 6 and summary["max_concurrent"] == 1


def test_request_on_an_existing_mesh_with_default_rhs(mfx):
    """A request may name a Mesh instead of an octree description; without a right-hand side function
    b = 1 (then distributed).  The result matches mfx_solve on the same data."""
    srv = mfx.Server(budget_bytes=4 << 30, max_slots=2, chunk=8)
    try:
        mesh = mfx.Mesh.structured_box(5, 5, 5, synthetic.deformed_vertices(5, 5, 5))
        t = srv.submit(3, mesh=mesh, coef_kind=mfx.COEF_TRIG, coef_par=(1.0, 0.5))
        info = wait_all(srv, [t], mfx)[t]
        assert info["state"] == mfx.REQ_DONE and info["stats"]["status"] == 0
        assert info["t_submit"] <= info["t_admit"] <= info["t_ready"] <= info["t_done"]
        x = srv.result(t)
        op = mfx.Operator(mesh, 3, mfx.COEF_TRIG, (1.0, 0.5))
        b = torch.ones(op.n_dofs, dtype=torch.float64, device="cuda")
        op.distribute(b)
        xa = torch.zeros_like(b)
        assert op.solve(b, xa, tol=1e-10, mixed=True)["status"] == 0
        xa = xa.cpu().numpy()
        assert np.linalg.norm(x - xa) <= 1e-9 * np.linalg.norm(xa)
        srv.retire(t)
        with pytest.raises(mfx.MfxError):
            srv.poll(t)  # retired tickets are forgotten
    finally:
        srv.close()


def test_cancel_retire_and_policy(mfx):
    """One slot: the first request runs, the rest queue.  A queued request cancels at once, a running
    one at the scheduler's next step; retiring an unfinished request is refused (MFX_EBUSY).  With the
    smallest-first policy the queued requests are admitted by estimated size."""
    leaves_big = synthetic.octree_leaves(6, 2, np.array([0.5, 0.5, 0.5]), 0.3)
    leaves_small = synthetic.octree_leaves(2, 1, np.array([0.3, 0.3, 0.3]), 0.2)
    srv = mfx.Server(budget_bytes=64 << 30, max_slots=1, chunk=4, policy=mfx.ADMIT_SMALLEST_FIRST)
    try:
        t_run = srv.submit(4, leaves=leaves_big, n_coarse=6, max_it=100000)
        t_big = srv.submit(3, leaves=leaves_big, n_coarse=6)
        t_small = srv.submit(2, leaves=leaves_small, n_coarse=2)
        t_cancel = srv.submit(1, leaves=leaves_small, n_coarse=2)
        srv.cancel(t_cancel)
        assert srv.poll(t_cancel)["state"] == mfx.REQ_CANCELLED
        with pytest.raises(mfx.MfxError) as e:
            srv.retire(t_big)  # still queued
        assert e.value.code == mfx.EBUSY
        # wait until the first request runs, then cancel it
        t0 = time.perf_counter()
        while srv.poll(t_run)["state"] < mfx.REQ_RUNNING:
            assert time.perf_counter() - t0 < 60
            time.sleep(0.001)
        srv.cancel(t_run)
        infos = wait_all(srv, [t_run, t_big, t_small], mfx)
        assert infos[t_run]["state"] in (mfx.REQ_CANCELLED, mfx.REQ_DONE)
        assert infos[t_big]["state"] == mfx.REQ_DONE and infos[t_small]["state"] == mfx.REQ_DONE
        assert infos[t_small]["t_admit"] < infos[t_big]["t_admit"]  # smallest first
        for t in (t_run, t_big, t_small, t_cancel):
            srv.retire(t)
        st = srv.stats()
        assert st["retired"] == 4 and st["bytes_in_use"] == 0 and st["max_concurrent"] == 1
    finally:
        srv.close()
