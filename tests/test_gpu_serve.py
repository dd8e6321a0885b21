"""Serving loop: requests admitted while others run (continuous batching), each result equal to the
same problem solved alone within 1e-9 relative."""
import numpy as np
import pytest

from paper_1910_13247_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_served_results_equal_standalone_solves():
    from paper_1910_13247_gb300 import build, mfx, serve
    build.build()
    reqs = serve.make_requests(10, rate=400.0, seed=11, size_range=(1e3, 4e4))
    server = serve.Server(budget_bytes=8 << 30, max_slots=4, chunk=8)
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
        xa, xs = x.cpu().numpy(), req.result.cpu().numpy()
        assert np.linalg.norm(xs - xa) <= 1e-9 * np.linalg.norm(xa), req.rid


def test_admission_respects_the_memory_budget():
    from paper_1910_13247_gb300 import build, serve
    build.build()
    reqs = serve.make_requests(6, rate=1000.0, seed=12, size_range=(2e3, 2e4))
    # a budget below any single request still admits one at a time (never more than one active)
    server = serve.Server(budget_bytes=1, max_slots=4, chunk=8)
    summary = server.run(reqs)
    assert summary["completed"] == 6 and summary["max_concurrent"] == 1
