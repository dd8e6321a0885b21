"""Continuous-batching solve server on top of the batch engine (mfx_batch_*).

Requests are Poisson solves on adaptively refined (octree) meshes.  The loop
admits arrived requests in arrival order while the device-memory budget
allows (operator data plus solver workspace, estimated before the operator
is built), adds each admitted request to a free slot of the batch, and then
runs scheduler ticks: one tick advances every active solve by a chunk of
inner iterations in one graph launch.  Requests that arrive while others are
running are admitted between ticks as slots and memory free up, so their
work overlaps with the running ones on the GPU.  Completed solves leave
their slot immediately and release their memory.

Latency = completion time - arrival time (queueing + setup + solve).
"""
import math
import time

import numpy as np

from . import mfx, synthetic


class Request:
    def __init__(self, rid, arrival, degree, nb, leaves, seed):
        self.rid = rid
        self.arrival = arrival
        self.degree = degree
        self.nb = nb
        self.leaves = leaves
        self.seed = seed
        self.latency = None
        self.t_admit = None       # seconds from the start: admitted (set-up begins)
        self.t_ready = None       # set-up done, solve added to the batch
        self.setup_s = None       # set-up duration on its worker thread
        self.status = None
        self.n_dofs = None
        self.iterations = None


def bytes_estimate(n_cells, n_dofs, degree):
    """Device bytes of an operator and its solver workspace (FP64 + FP32 data)."""
    nq = n_cells * (degree + 1) ** 3
    return nq * (6 * 8 + 6 * 4 + 8) + n_cells * (degree + 1) ** 3 * 4 + n_dofs * (9 * 8 + 9 * 4 + 2 * 8 + 8 + 4 + 1)


def make_requests(n, rate=200.0, seed=5, size_range=(1e3, 1e7), max_fine=128):
    """Seeded request stream: exponential inter-arrival times (Poisson process of the given rate),
    degree uniform in 1..8, target size log-uniform in size_range, 1-3 refinement levels inside a
    seeded ball.  The coarse grid n_b^3 is the one whose estimated size is closest to the target,
    with n_b 2^levels <= max_fine (the generator's voxel limit), so the largest targets are clamped."""
    g = synthetic.rng(seed)
    t = 0.0
    reqs = []
    for i in range(n):
        t += float(g.exponential(1.0 / rate))
        k = int(g.integers(1, 9))
        target = math.exp(g.uniform(math.log(size_range[0]), math.log(size_range[1])))
        levels = int(g.integers(1, 4))
        center = g.uniform(0.2, 0.8, size=3)
        radius = float(g.uniform(0.15, 0.35))
        frac = min(1.0, 4.0 / 3.0 * math.pi * radius ** 3)
        per_coarse = (1.0 + frac * (8 ** levels - 1)) * k ** 3
        nb = int(round((target / per_coarse) ** (1.0 / 3.0)))
        nb = max(2, min(nb, max_fine >> levels))
        leaves = synthetic.octree_leaves(nb, levels, center, radius)
        reqs.append(Request(i, t, k, nb, leaves, seed * 100000 + i))
    return reqs


class Server:
    """Admission by memory budget, operator set-up on a background thread, and independent stepping of
    all active solves (mfx_batch_advance): each solve takes its next step as soon as its previous one
    has finished, so small requests are not held back by large ones."""

    def __init__(self, budget_bytes=64 << 30, max_slots=32, chunk=16, tol=1e-10):
        self.budget = budget_bytes
        self.batch = mfx.Batch(max_slots, chunk=chunk)
        self.max_slots = max_slots
        self.tol = tol

    @staticmethod
    def _setup(req):
        # runs on a set-up thread, on a stream of its own: no device-wide synchronisation, which
        # would collide with the graph captures of the serving thread
        import torch
        t0 = time.perf_counter()
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            mesh = mfx.Mesh.octree(req.nb, req.nb, req.nb, req.leaves)
            op = mfx.Operator(mesh, req.degree, stream=stream)
            op.prepare_solver()  # workspace here, not in the serving thread's batch.add
            b = torch.from_numpy(synthetic.gaussian_vector(op.n_dofs, req.seed)).pin_memory().to(
                "cuda", non_blocking=True)
            op.distribute(b, stream=stream)  # right-hand side on the free DoFs only
            x = torch.zeros_like(b)
        stream.synchronize()
        req.setup_s = time.perf_counter() - t0
        return op, b, x

    def run(self, requests, time_limit=None):
        """Serve the requests (arrival times relative to the start); returns a summary dict."""
        import concurrent.futures as cf

        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        queue = []        # arrived, not admitted (arrival order)
        setting_up = {}   # future -> (req, estimated bytes)
        active = {}       # slot -> (req, op, b, x, bytes)
        used = 0
        done = []
        max_active = 0
        pool = cf.ThreadPoolExecutor(max_workers=4)
        start = time.perf_counter()
        while pending or queue or active or setting_up:
            now = time.perf_counter() - start
            if time_limit is not None and now > time_limit:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            # admission in arrival order, by memory budget and free slots
            while queue and len(active) + len(setting_up) < self.max_slots:
                req = queue[0]
                n_cells = len(req.leaves)
                est = bytes_estimate(n_cells, n_cells * req.degree ** 3 * 2, req.degree)
                if (active or setting_up) and used + est > self.budget:
                    break
                queue.pop(0)
                used += est
                req.t_admit = time.perf_counter() - start
                setting_up[pool.submit(self._setup, req)] = (req, est)
            for fut in [f for f in setting_up if f.done()]:
                req, est = setting_up.pop(fut)
                op, b, x = fut.result()
                nbytes = op.info()["bytes_device"] + op.n_dofs * (9 * 8 + 9 * 4 + 16)
                used += nbytes - est
                slot = self.batch.add(op, b, x, tol=self.tol, mixed=True)
                req.t_ready = time.perf_counter() - start
                active[slot] = (req, op, b, x, nbytes)
                req.n_dofs = op.n_dofs
            max_active = max(max_active, len(active))
            if active:
                self.batch.advance()
                t_now = time.perf_counter() - start
                for slot in list(active):
                    fin, st = self.batch.poll(slot)
                    if fin:
                        req, op, b, x, nbytes = active.pop(slot)
                        req.latency = t_now - req.arrival
                        req.status = st["status"]
                        req.iterations = st["inner_iterations"]
                        req.result = x
                        self.batch.release(slot)
                        op.release()  # its slot reported done: free in stream order, no device-wide wait
                        used -= nbytes
                        done.append(req)
            time.sleep(0.0002)
        pool.shutdown(wait=True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - start
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        # where the latency goes: waiting for admission, set-up (host tables, geometry, diagonal),
        # and the solve itself (from joining the batch to completion)
        wait = np.array([r.t_admit - r.arrival for r in done]) if done else np.zeros(1)
        setup = np.array([r.setup_s for r in done]) if done else np.zeros(1)
        solve = np.array([r.arrival + r.latency - r.t_ready for r in done]) if done else np.zeros(1)
        span = max(r.arrival for r in requests) if requests else 0.0
        return {
            "requests": len(requests), "completed": len(done), "wall_seconds": wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(done) / wall if wall > 0 else 0.0,
            "offered_rate_per_s": len(requests) / span if span > 0 else float("inf"),
            "max_concurrent": max_active, "statuses": sorted({r.status for r in done}),
            "p50_admission_wait_s": float(np.percentile(wait, 50)), "p50_setup_s": float(np.percentile(setup, 50)),
            "total_setup_s": float(setup.sum()), "p50_solve_s": float(np.percentile(solve, 50)),
            "dofs_min": int(min(r.n_dofs for r in done)) if done else 0,
            "dofs_max": int(max(r.n_dofs for r in done)) if done else 0,
            "degrees": sorted({r.degree for r in done}),
        }
