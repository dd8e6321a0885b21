"""Serving workload: Poisson solves on adaptively refined (octree) meshes arriving as a Poisson process,
served by the library's native solve server (mfx_server_*, continuous batching).

The server admits arrived requests in arrival order while the device-memory budget allows (operator
data plus solver workspace, estimated before the operator is built), builds each admitted request's
operator on a set-up thread, and adds it to a free slot of its batch, where every running solve takes
its next chunk of inner iterations as soon as its previous one has finished.  Requests that arrive
while others are running are admitted as slots and memory free up, so their work overlaps with the
running ones on the GPU.

Latency = completion time - arrival time (queueing + set-up + solve).
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


def make_requests(n, rate=200.0, seed=5, size_range=(1e3, 1e7), max_fine=512):
    """Seeded request stream: exponential inter-arrival times (Poisson process of the given rate),
    degree uniform in 1..8, target size log-uniform in size_range, 1-3 refinement levels inside a
    seeded ball.  The coarse grid n_b^3 is the one whose estimated size is closest to the target,
    with n_b 2^levels <= max_fine (the generator's finest voxel grid, 512^3 by default: targets up to
    10^7 DoFs are reached at every degree and level count)."""
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
    """Drives the library's native solve server (mfx_server_*): requests are submitted at their arrival
    times; the library admits them by memory budget, builds their operators on its set-up threads and
    steps every running solve on its scheduler thread, each solve taking its next step as soon as its
    previous one has finished (small requests are not held back by large ones).  This class only
    submits, polls and collects results."""

    def __init__(self, budget_bytes=64 << 30, max_slots=32, chunk=16, tol=1e-10, setup_threads=4,
                 policy=mfx.ADMIT_FIFO, keep_results=False):
        self.budget = budget_bytes
        self.max_slots = max_slots
        self.chunk = chunk
        self.tol = tol
        self.setup_threads = setup_threads
        self.policy = policy
        self.keep_results = keep_results

    def run(self, requests, time_limit=None):
        """Serve the requests (arrival times relative to the start); returns a summary dict."""
        srv = mfx.Server(self.budget, self.max_slots, self.chunk, self.setup_threads, self.policy)
        pending = sorted(requests, key=lambda r: r.arrival)
        outstanding = {}  # ticket -> (request, client time of submission)
        done = []
        start = time.perf_counter()
        try:
            while pending or outstanding:
                now = time.perf_counter() - start
                if time_limit is not None and now > time_limit:
                    for t in outstanding:
                        srv.cancel(t)
                    break
                while pending and pending[0].arrival <= now:
                    req = pending.pop(0)
                    seed = req.seed
                    t = srv.submit(req.degree, leaves=req.leaves, n_coarse=req.nb, tol=self.tol, mixed=True,
                                   rhs=lambda n, seed=seed: synthetic.gaussian_vector(n, seed))
                    outstanding[t] = (req, time.perf_counter() - start)
                for t in list(outstanding):
                    info = srv.poll(t)
                    if info["state"] < mfx.REQ_DONE:
                        continue
                    req, t_sub = outstanding.pop(t)
                    offset = t_sub - info["t_submit"]  # client clock minus server clock
                    req.latency = info["t_done"] + offset - req.arrival
                    req.t_admit = info["t_admit"] + offset
                    req.t_ready = info["t_ready"] + offset
                    req.setup_s = info["setup_seconds"]
                    req.status = info["stats"]["status"] if info["state"] == mfx.REQ_DONE else -100 - info["state"]
                    req.iterations = info["stats"]["inner_iterations"]
                    req.n_dofs = info["n_dofs"]
                    if self.keep_results and info["state"] == mfx.REQ_DONE:
                        req.result = srv.result(t)
                    srv.retire(t)
                    done.append(req)
                time.sleep(0.0005)
            st = srv.stats()
        finally:
            srv.close()
        wall = time.perf_counter() - start
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        # where the latency goes: waiting for admission, set-up (mesh, tables, geometry, diagonal,
        # workspace, right-hand side) and the solve itself (from joining the batch to completion)
        wait = np.array([r.t_admit - r.arrival for r in done]) if done else np.zeros(1)
        setup = np.array([r.setup_s for r in done]) if done else np.zeros(1)
        solve = np.array([r.arrival + r.latency - r.t_ready for r in done]) if done else np.zeros(1)
        span = max(r.arrival for r in requests) if requests else 0.0
        return {
            "requests": len(requests), "completed": len(done), "wall_seconds": wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(done) / wall if wall > 0 else 0.0,
            "offered_rate_per_s": len(requests) / span if span > 0 else float("inf"),
            "max_concurrent": int(st["max_concurrent"]), "statuses": sorted({r.status for r in done}),
            "p50_admission_wait_s": float(np.percentile(wait, 50)), "p50_setup_s": float(np.percentile(setup, 50)),
            "total_setup_s": float(setup.sum()), "p50_solve_s": float(np.percentile(solve, 50)),
            "dofs_min": int(min(r.n_dofs for r in done)) if done else 0,
            "dofs_max": int(max(r.n_dofs for r in done)) if done else 0,
            "degrees": sorted({r.degree for r in done}),
            "runtime": "native (mfx_server_*: set-up threads, scheduler thread)",
        }
