"""Benchmark: matrix-free Q_k Laplacian vmult on GB300.

Workload: 64^3 hexahedra of the unit cube deformed by
x -> x + 0.05 sin(pi x) sin(pi y) sin(pi z) (every component), Q4 on
Gauss-Lobatto nodes, 5-point Gauss quadrature per direction, coefficient
a = 1 + 0.5 sin(2 pi x) cos(2 pi y) z, homogeneous Dirichlet boundary,
16,974,593 DoFs, seeded uniform[-1, 1] input vectors (synthetic).

One step = one operator application (vmult) in FP32 (the headline) --
the FP64 vmult, the FP64 and mixed solves and the end-to-end path are
reported beside it.  Every step reads more than the 129 MB L2 (about
0.92 GB per FP32 step), so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs the same workload on its own GPU
(independent replicas, weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, K_DEG = 64, 4
# More hardware work queues than the default 8, so that the many streams of the batch engine and the
# serving loop (one per problem, plus the set-up threads' streams) do not falsely serialise behind each
# other.  Read when the CUDA context is created, so it is set before torch touches the GPU.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "matrix-free vmult GDoF/s (FP64 vs FP32 mixed) and % HBM peak; solve p50/p99 latency"
WORKLOAD = "64^3 deformed unit cube, Q4 GLL, 5-pt Gauss, a=1+0.5 sin(2pi x)cos(2pi y)z, Dirichlet"


# DRAM traffic of one FP32 vmult launch on the 64^3 Q4 workload, from the ncu capture summarised in
# profiles/vmult_fp32_f5_staged_q4_48cube.md (48^3 case, five-phase kernel with the staged metric, 8 cells per
# batch; 412.85 MB read + written, scaled by cells to 64^3).  Valid only for that kernel, batch size and the
# kernel sources it was taken from: anything else reports null.
TRAFFIC_BYTES = 978.4e6
TRAFFIC_KERNEL = (3, 8)  # (structured_kernel, cells_per_block): five-phase, staged metric, 8 cells per batch
TRAFFIC_SOURCES = {"vmult_brick_f5.cuh": "4f7d5a2e9488aa25", "vmult_brick_tma2.cuh": "0991fee5e2c07a72",
                   "vmult_brick_tma.cuh": "25984cf632f8c607", "vmult_brick.cuh": "d4348f1901d2181e",
                   "vmult.cuh": "a6088d02147ee108", "vmult_launch.cuh": "81978a63b553fbee"}
KERNEL_NAMES = {1: "brick_vmult_tma2_kernel (ten phases)", 2: "brick_vmult_f5_kernel (five phases, metric from L2)",
                3: "brick_vmult_f5_kernel (five phases, metric staged in shared memory)"}


def measured_traffic(nx, k, cells_per_block, kernel):
    import hashlib
    if (nx, k) != (NX, K_DEG) or (kernel, cells_per_block) != TRAFFIC_KERNEL:
        return None
    csrc = os.path.join(ROOT, "paper_1910_13247_gb300", "csrc")
    for name, digest in TRAFFIC_SOURCES.items():
        with open(os.path.join(csrc, name), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != digest:
                return None
    return TRAFFIC_BYTES


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bytes_per_vmult(n_dofs, n_cells, k, s):
    """Algorithmic bytes: src read + dst write (2 s N) and the 6-entry metric per quadrature point."""
    return 2 * s * n_dofs + 6 * s * n_cells * (k + 1) ** 3


def aggregate_ranks(elapsed_ms, units_per_rank, dist=None, device=None):
    """Whole-job throughput of replicas: the slowest rank's time, the work of all ranks.

    Returns (max elapsed ms over ranks, total units / that time in units per second)."""
    import torch
    world = 1
    t = float(elapsed_ms)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        v = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
    return t, world * units_per_rank / (t * 1e-3)


THROTTLE_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clocks):
    """A timed region is not a valid measurement if its clock record shows a hardware or thermal slowdown,
    or SM clocks well below their maximum with no reason at all (a leftover clock lock); a power cap is
    kept (it is noted in the record)."""
    if not clocks:
        return False
    if any(r in THROTTLE_REASONS for r in clocks["reasons"]):
        return True
    return clocks["sm_max_mhz"] > 0 and clocks["sm_mhz"] < 0.85 * clocks["sm_max_mhz"] and not clocks["reasons"]


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds=12.0, sub=12, one_core=True, steps=None, warmup=0):
    """The FP64 oracle (assembled CSR SpMV, OpenMP) on a sub-mesh of the same workload.

    Runs SpMVs for `seconds`, or, with `steps` given, `warmup` untimed SpMVs and then exactly `steps` timed
    ones (one step = one SpMV over the sub-mesh)."""
    import numpy as np
    from oracle import fem, mesh
    from paper_1910_13247_gb300 import synthetic
    verts = synthetic.deformed_vertices(sub, sub, sub)
    om = mesh.structured_mesh(sub, sub, sub, K_DEG, verts)
    t0 = time.perf_counter()
    K = fem.assemble(om, K_DEG + 1, fem.COEF_TRIG, (1.0, 0.5))
    t_asm = time.perf_counter() - t0
    A = fem.CSR(K)
    x = synthetic.uniform_vector(om.n_dofs, 1)
    y = np.zeros(om.n_dofs)
    A(x, y)
    if steps is not None:
        for _ in range(warmup):
            A(x, y)
        t0 = time.perf_counter()
        for _ in range(steps):
            A(x, y)
        reps = steps
        seconds = time.perf_counter() - t0
    else:
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            A(x, y)
            reps += 1
        seconds = time.perf_counter() - t0
    dt = seconds / reps
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if one_core and cores > 1:
        # the same SpMV on one core (a fresh process: the OpenMP team size is fixed at start)
        env = dict(os.environ, OMP_NUM_THREADS="1")
        code = ("import json, bench; print(json.dumps(bench.cpu_baseline(seconds=%r, sub=%d, one_core=False)))"
                % (max(2.0, seconds / 4), sub))
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
        one = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 and r.stdout.strip() else None
    else:
        one = None
    return {"value": om.n_dofs / dt / 1e9, "unit": "GDoF/s", "cores": cores, "kind": "oracle", "ms_per_spmv": dt * 1e3,
            "one_core_value": one["value"] if one else None,
            "sample": f"FP64 CSR SpMV of the oracle-assembled operator on a {sub}^3-cell sub-mesh of the same "
                      f"workload ({om.n_dofs} DoFs, {K.nnz} nonzeros), {reps} SpMVs over {seconds:.1f} s; "
                      f"assembly ({t_asm:.1f} s) excluded"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # one step = one oracle SpMV over the sub-mesh (a few ms on the host cores), so K steps stay bounded
    cb = cpu_baseline(steps=args.steps, warmup=args.warmup)
    line = {"metric": METRIC, "value": cb["value"], "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cb["ms_per_spmv"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_dofs": (NX * K_DEG + 1) ** 3, "n_cells": NX ** 3, "degree": K_DEG,
                       "n_q_1d": K_DEG + 1, "step": "one FP64 oracle SpMV over a 12^3-cell sample of the workload",
                       "parallelism": "host cores"},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mfx")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-solve", action="store_true", help="skip the solve measurements")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 96^3 Q3 mixed-precision solve")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-problem batched solve")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run")
    ap.add_argument("--no-sipg", action="store_true", help="skip the SIPG DG vmult and multigrid solve")
    ap.add_argument("--sipg-dims", type=int, nargs=3, default=[128, 64, 64],
                    help="cells of the SIPG hyper-rectangle (profiling on smaller cases)")
    ap.add_argument("--sipg-vmult-only", action="store_true", help="SIPG: time the vmult only, no multigrid solve")
    ap.add_argument("--sipg-degree", type=int, default=4, help="SIPG polynomial degree (the paper's benchmark: 4)")
    ap.add_argument("--no-octree", action="store_true", help="skip the octree vmult (hanging nodes)")
    ap.add_argument("--octree-degree", type=int, default=4, help="degree of the octree vmult measurement")
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--nx", type=int, default=NX, help="cells per direction (profiling on smaller cases)")
    ap.add_argument("--degree", type=int, default=K_DEG)
    ap.add_argument("--cells-per-block", type=int, default=0,
                    help="fix the structured kernel's cells per batch (0: autotuned at operator creation)")
    ap.add_argument("--fp32-kernel", type=int, default=0,
                    help="fix the structured FP32 kernel (1 ten-phase, 2 five-phase, 3 five-phase staged; 0: autotuned)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_1910_13247_gb300 import build, mfx, synthetic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    stream = torch.cuda.current_stream()

    nx, kdeg = args.nx, args.degree
    verts = synthetic.deformed_vertices(nx, nx, nx)
    mesh = mfx.Mesh.structured_box(nx, nx, nx, verts)
    op = mfx.Operator(mesh, kdeg, mfx.COEF_TRIG, (1.0, 0.5), cells_per_block=args.cells_per_block,
                      structured_kernel=args.fp32_kernel)
    N, C = op.n_dofs, op.n_cells
    x64 = torch.tensor(synthetic.uniform_vector(N, 1), device="cuda")
    x32 = x64.float()
    y64, y32 = torch.empty_like(x64), torch.empty_like(x32)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()

    # warm-up
    for _ in range(max(3, args.warmup)):
        op.vmult(x32, y32)
    op.vmult(x64, y64)
    barrier()

    def timed_region():
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)  # nvidia-smi's first sample
        # untimed load right before the timed steps, so that the clock samples (every 100 ms) see the
        # GPU under this workload even when the K timed steps take only a few milliseconds
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < 0.4:
            for _ in range(20):
                op.vmult(x32, y32)
            torch.cuda.synchronize()
        # timed region: K FP32 vmults, each bracketed by events on the launching stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            op.vmult(x32, y32)
            ev[i][1].record(stream)
        t_end.record(stream)
        barrier()
        return t_start, t_end, ev, sampler.stop()

    t_start, t_end, ev, clocks = timed_region()
    first_clocks = None
    # a region that saw a slowdown or a clock lock is measured once more (the decision is collective)
    rejected_twice = False
    if max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0) > 0.0:
        first_clocks = clocks
        t_start, t_end, ev, clocks = timed_region()
        rejected_twice = max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0) > 0.0
    total_ms, units_per_s = aggregate_ranks(t_start.elapsed_time(t_end), N * args.steps, dist, "cuda")
    per_launch = [a.elapsed_time(b) for a, b in ev]
    ms32 = statistics.mean(per_launch)
    q32 = statistics.quantiles(per_launch, n=10) if len(per_launch) >= 10 else [ms32] * 9
    ms_per_step = total_ms / args.steps
    value = units_per_s / 1e9

    hbm, peak_kind = peaks()
    b32 = bytes_per_vmult(N, C, kdeg, 4)
    b64 = bytes_per_vmult(N, C, kdeg, 8)
    achieved = b32 / (ms32 * 1e-3) / 1e9

    # FP64 vmult (ALU-bound on GB300: reported with its own roofline)
    reps64 = max(10, min(200, args.steps // 10))
    ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps64)]
    for i in range(reps64):
        ev64[i][0].record(stream)
        op.vmult(x64, y64)
        ev64[i][1].record(stream)
    torch.cuda.synchronize()
    per64 = [a.elapsed_time(b) for a, b in ev64]
    ms64 = statistics.mean(per64)
    q64 = statistics.quantiles(per64, n=10) if len(per64) >= 10 else [ms64] * 9

    # end to end through the C-ABI with host buffers (mfx_vmult_host): every step uploads its input from
    # pinned host memory, applies the operator and downloads the result; the library pipelines the
    # steps (upload of i + 1, vmult of i, download of i - 1 overlap).  Two pinned inputs and two pinned
    # outputs alternate; host-timed around the call, which returns when every result is on the host.
    h_in = [torch.empty(N, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    for h in h_in:
        h.copy_(x32.cpu())
    h_out = [torch.empty(N, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    n_e2e = 100  # fixed: the pipeline's fill and drain are amortised the same way whatever --steps is
    srcs = [h_in[i % 2] for i in range(n_e2e)]
    dsts = [h_out[i % 2] for i in range(n_e2e)]
    op.vmult_host(srcs[:2], dsts[:2])  # warm-up (streams, staging pool)
    barrier()
    t0 = time.perf_counter()
    op.vmult_host(srcs, dsts)
    barrier()
    ms_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3 / n_e2e)
    # same result as the device-resident run (atomic scatter order may change the last bits)
    for h in h_out:
        assert torch.allclose(h, y32.cpu(), rtol=0, atol=1e-5 * y32.abs().max().item())

    line = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if (nx, kdeg) == (NX, K_DEG) else f"{nx}^3 cells, Q{kdeg} (profiling case)",
                   "n_dofs": N, "n_cells": C, "degree": kdeg, "n_q_1d": kdeg + 1,
                   "cells_per_block": op.info()["cells_per_block"], "fp32_kernel": op.info()["structured_kernel"],
                   "step": "one FP32 vmult", "l2": "inputs larger than L2 (%.2f GB read+written per step)" % (b32 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": measured_traffic(nx, kdeg, op.info()["cells_per_block"], op.info()["structured_kernel"]),
                     "peak_kind": peak_kind,
                     "kernel": "FP32 vmult (init_rows_kernel + %s, %d cells per batch), timed together"
                               % (KERNEL_NAMES.get(op.info()["structured_kernel"], "per-cell kernel"),
                                  op.info()["cells_per_block"]),
                     "algorithmic_bytes": b32,
                     # secondary model: coefficient per q-point and vertices instead of the stored metric
                     "algorithmic_bytes_minimal": 2 * 4 * N + 4 * C * (kdeg + 1) ** 3 + 24 * C},
        "e2e": {"value": world * N / (ms_e2e * 1e-3) / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 4 * N, "ms_per_step": ms_e2e, "steps": n_e2e,
                "call": "mfx_vmult_host (pinned host vectors, upload / vmult / download pipelined)"},
        "gpu_launches": 2 * args.steps,
        "fp64": {"gdofs": N / (ms64 * 1e-3) / 1e9, "ms": ms64, "algorithmic_bytes": b64,
                 "hbm_frac": b64 / (ms64 * 1e-3) / 1e9 / hbm,
                 "launch_ms": {"median": statistics.median(per64), "p10": q64[0], "p90": q64[-1], "reps": reps64}},
        "fp32_ms_per_launch": ms32,
        "fp32_launch_ms": {"median": statistics.median(per_launch), "p10": q32[0], "p90": q32[-1],
                           "reps": len(per_launch)},
    }
    if clocks:
        line["clocks"] = clocks
    if first_clocks:
        line["clocks_first_run_rejected"] = first_clocks
        line["clocks_rejected_twice"] = rejected_twice

    if not args.no_solve:
        line["solve"] = solve_measurements(mfx, synthetic, torch, np)
        if not args.no_mixed:
            line["solve"]["mixed_96x96x96_q3"] = mixed_solve_measurement(mfx, synthetic, torch, np)
        if not args.no_batch:
            line["batched"] = batched_measurement(mfx, synthetic, torch, np)
        if not args.no_serve:
            line["serving"] = serving_measurement(args.serve_requests)
        if not args.no_octree:
            line["octree"] = octree_measurement(mfx, synthetic, torch, args.octree_degree)
            # the same refinement on 32^3 coarse cells (17.5M DoFs at Q4): the kernels at a serving-size mesh
            line["octree"]["large"] = octree_measurement(mfx, synthetic, torch, args.octree_degree, nb=32, fp64=False)
            # the same leaves on the undeformed cube with a constant coefficient (the serving requests' form)
            line["octree"]["large_box"] = octree_measurement(mfx, synthetic, torch, args.octree_degree, nb=32,
                                                             fp64=False, box=True)
        if not args.no_sipg:
            line["sipg"] = sipg_measurement(mfx, synthetic, torch, np, tuple(args.sipg_dims), k=args.sipg_degree,
                                            solve=not args.sipg_vmult_only)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def solve_measurements(mfx, synthetic, torch, np):
    """Latency of the 8^3 Q2 Poisson Jacobi-PCG solve (p50/p99 over repeated solves)."""
    out = {}
    m = mfx.Mesh.structured_box(8, 8, 8)
    op = mfx.Operator(m, 2, mfx.COEF_CONSTANT, (1.0, 0.0))
    n3 = 27
    xq = torch.empty(op.n_cells * n3 * 3, dtype=torch.float64, device="cuda")
    op.quadrature_points(xq)
    X = xq.view(-1, 3)
    fq = 3 * np.pi ** 2 * torch.sin(np.pi * X[:, 0]) * torch.sin(np.pi * X[:, 1]) * torch.sin(np.pi * X[:, 2])
    b = torch.empty(op.n_dofs, dtype=torch.float64, device="cuda")
    op.rhs(fq.contiguous(), b)
    x = torch.zeros_like(b)
    lat, its = [], 0
    for i in range(23):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op.solve(b, x, tol=1e-10)
        lat.append((time.perf_counter() - t0) * 1e3)
        its = st["iterations"]
    lat = sorted(lat[3:])
    out["poisson_8x8x8_q2_jacobi_pcg"] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                           "iterations": its, "rel_residual": st["rel_residual"], "runs": len(lat)}
    # the 8^3 Q2 operator fits in L2: its vmult is reported as latency
    stream = torch.cuda.current_stream()
    for name, dt in (("vmult_8x8x8_q2_fp64_us", torch.float64), ("vmult_8x8x8_q2_fp32_us", torch.float32)):
        xs = torch.tensor(synthetic.uniform_vector(op.n_dofs, 1), device="cuda", dtype=dt)
        ys = torch.empty_like(xs)
        for _ in range(10):
            op.vmult(xs, ys)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
        for e0, e1 in evs:
            e0.record(stream)
            op.vmult(xs, ys)
            e1.record(stream)
        torch.cuda.synchronize()
        us = sorted(1e3 * a.elapsed_time(b) for a, b in evs)
        out[name] = {"median": us[len(us) // 2], "p10": us[len(us) // 10], "p90": us[(9 * len(us)) // 10],
                     "reps": len(us)}
    return out


def serving_measurement(n_requests, rate=200.0, seed=5):
    """Poisson arrivals (200/s) of octree Poisson solves, degree 1..8, sizes log-uniform in 1e3..1e7 DoFs,
    tol 1e-10, continuous batching under a 64 GB device-memory budget; operator set-up on host threads (all
    cores but two)."""
    from paper_1910_13247_gb300 import mfx, serve
    threads = max(4, (os.cpu_count() or 8) - 2)
    reqs = serve.make_requests(n_requests, rate=rate, seed=seed)
    server = serve.Server(budget_bytes=64 << 30, max_slots=32, chunk=16, setup_threads=threads)
    out = server.run(reqs, time_limit=240.0)
    out["budget_bytes"] = 64 << 30
    out["policy"] = "fifo"
    # the same stream admitted smallest-first (estimated device bytes): small requests stop queueing
    # behind large ones while the offered load exceeds capacity
    out["setup_threads"] = threads
    small = serve.Server(budget_bytes=64 << 30, max_slots=32, chunk=16, setup_threads=threads,
                         policy=mfx.ADMIT_SMALLEST_FIRST)
    alt = small.run(serve.make_requests(n_requests, rate=rate, seed=seed), time_limit=240.0)
    out["smallest_first"] = {key: alt[key] for key in ("p50_latency_s", "p99_latency_s", "solves_per_s", "wall_seconds",
                                                        "completed") if key in alt}
    return out


def batched_measurement(mfx, synthetic, torch, np, n_problems=64, seed=4):
    """64 independent Poisson problems (unit cube, N^3 cells with N uniform in [4, 32], degree uniform in 1..6,
    uniform[-1, 1] right-hand sides, FP32 inner / FP64 outer Jacobi-PCG to 1e-10) solved together in one graph
    launch (mfx_batch_run), and by host-driven ticks (mfx_batch_step), against the same solves run one after
    another."""
    g = synthetic.rng(seed)
    Ns = g.integers(4, 33, size=n_problems)
    ks = g.integers(1, 7, size=n_problems)
    ops, bs = [], []
    for i in range(n_problems):
        op = mfx.Operator(mfx.Mesh.structured_box(int(Ns[i]), int(Ns[i]), int(Ns[i])), int(ks[i]))
        b = torch.tensor(synthetic.uniform_vector(op.n_dofs, 1000 + i), device="cuda")
        op.distribute(b)
        ops.append(op)
        bs.append(b)
    total_dofs = sum(op.n_dofs for op in ops)
    # one after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_inner = 0
    for op, b in zip(ops, bs):
        st = op.solve(b, torch.zeros_like(b), tol=1e-10, mixed=True)
        seq_inner += st["inner_iterations"] * op.n_dofs
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    def together(one_launch):
        batch = mfx.Batch(n_problems, chunk=16)
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        slots = [batch.add(op, b, x, tol=1e-10, mixed=True) for op, b, x in zip(ops, bs, xs)]
        # one graph launch whose device-side loops decide when each problem stops, or host-driven ticks
        launches = 1 if one_launch and batch.run_once() else batch.run()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        dof_iters, worst, statuses = 0, 0.0, set()
        for op, s in zip(ops, slots):
            done, st = batch.poll(s)
            statuses.add(st["status"] if done else -99)
            dof_iters += st["inner_iterations"] * op.n_dofs
            worst = max(worst, st["rel_residual"])
        return t, launches, dof_iters, worst, sorted(statuses)

    t_batch, launches, dof_iters, worst, statuses = together(True)
    t_ticks, ticks, _, worst_ticks, statuses_ticks = together(False)
    chosen = {}
    for op, n_, k_ in zip(ops, Ns, ks):
        chosen.setdefault(f"k{int(k_)}", {})[int(n_)] = [op.info()["cells_per_block"], op.info()["structured_kernel"]]
    return {"problems": n_problems, "total_dofs": total_dofs, "seconds": t_batch, "graph_launches": launches,
            "mode": "one graph launch; per problem a device-decided WHILE loop (outer corrections, inner PCG)",
            "autotuned_cells_per_block_and_kernel": chosen,
            "dof_iterations_per_s": dof_iters / t_batch, "statuses": statuses, "max_rel_residual": worst,
            "sequential_seconds": t_seq, "speedup_over_sequential": t_seq / t_batch,
            "ticks_mode": {"seconds": t_ticks, "ticks": ticks, "statuses": statuses_ticks,
                           "max_rel_residual": worst_ticks, "speedup_over_sequential": t_seq / t_ticks},
            "sizes": {"N": [int(v) for v in Ns], "k": [int(v) for v in ks]}}


def mixed_solve_measurement(mfx, synthetic, torch, np):
    """96^3 deformed Q3 with the variable coefficient: FP64 Chebyshev(5)-Jacobi PCG versus FP32 PCG with the
    same preconditioner (to 1e-4) inside FP64 defect correction, both to a 1e-10 relative residual."""
    nx = 96
    m = mfx.Mesh.structured_box(nx, nx, nx, synthetic.deformed_vertices(nx, nx, nx))
    op = mfx.Operator(m, 3, mfx.COEF_TRIG, (1.0, 0.5))
    n = op.n_dofs
    b = torch.tensor(synthetic.gaussian_vector(n, 3), device="cuda")
    t = torch.tensor(synthetic.uniform_vector(n, 33), device="cuda")
    out = {"n_dofs": n}
    xs = {}
    for name, mixed in (("fp64", False), ("mixed", True)):
        # constrained rows of b are zero: the right-hand side lives on the free DoFs
        x = torch.zeros_like(b)
        bb = b.clone()
        op.distribute(bb)   # Dirichlet entries -> 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op.solve(bb, x, tol=1e-10, precond=mfx.PRECOND_CHEBYSHEV, cheb_degree=5, mixed=mixed,
                      inner_tol=1e-4, lanczos_start=t)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        xs[name] = x
        out[name] = {"seconds": dt, "status": st["status"], "iterations": st["iterations"],
                     "inner_iterations": st["inner_iterations"], "rel_residual": st["rel_residual"],
                     "lambda_max": st["lambda_max"]}
    out["speedup_mixed_over_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    out["rel_difference_mixed_vs_fp64"] = float((xs["mixed"] - xs["fp64"]).norm() / xs["fp64"].norm())
    # the paper's large-scale solver: PCG with the geometric multigrid V-cycle (Chebyshev(6) smoothing on
    # 96, 48, 24, 12, 6 cells per direction, exact solve on 3^3 cells), FP64 and mixed precision
    del op
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = mfx.Multigrid(m, 3, mfx.COEF_TRIG, (1.0, 0.5), smoother_degree=6)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    fine = g.fine
    for name, mixed in (("mg_fp64", False), ("mg_mixed", True)):
        x = torch.zeros_like(b)
        bb = b.clone()
        fine.distribute(bb)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.solve(bb, x, tol=1e-10, mixed=mixed, inner_tol=1e-4)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "status": st["status"], "iterations": st["iterations"],
                     "inner_iterations": st["inner_iterations"], "rel_residual": st["rel_residual"],
                     "rel_difference_vs_fp64_cheb": float((x - xs["fp64"]).norm() / xs["fp64"].norm())}
    out["mg_levels"] = g.n_levels
    out["mg_setup_seconds"] = setup
    out["speedup_mg_mixed_over_cheb_mixed"] = out["mixed"]["seconds"] / out["mg_mixed"]["seconds"]
    return out


def octree_bytes(n_dofs, n_cells, k, s, box=False):
    """Algorithmic bytes of an octree vmult: src read and dst written, the 6-entry metric per quadrature
    point (box cells: 3 entries per cell), the int32 cell DoF table; the hanging constraints' words and
    coarse-DoF lists are left out (they are a few bytes per hanging cell)."""
    n3 = (k + 1) ** 3
    metric = 3 * s * n_cells if box else 6 * s * n_cells * n3
    return 2 * s * n_dofs + metric + 4 * n_cells * n3


def octree_measurement(mfx, synthetic, torch, k=4, nb=16, levels=2, fp64=True, box=False):
    """FP32 and FP64 vmult on an octree refined twice inside a ball (hanging nodes; the serving
    workload's mesh family): nb^3 coarse cells of the deformed cube, the variable coefficient; box=True:
    the undeformed cube and a constant coefficient (the serving requests' operator: every cell an
    axis-aligned box, the FP32 metric one diagonal per cell)."""
    leaves = synthetic.octree_leaves(nb, levels, (0.5, 0.45, 0.55), 0.3)
    if box:
        op = mfx.Operator(mfx.Mesh.octree(nb, nb, nb, leaves), k)
    else:
        mesh = mfx.Mesh.octree(nb, nb, nb, leaves, synthetic.deformed_vertices(nb, nb, nb))
        op = mfx.Operator(mesh, k, mfx.COEF_TRIG, (1.0, 0.5))
    info = op.info()
    n = op.n_dofs
    hbm, peak_kind = peaks()
    out = {"workload": "octree, %d^3 coarse cells refined %d times in a ball, Q%d%s"
                       % (nb, levels, k, ", undeformed, constant coefficient" if box else ""), "n_dofs": n,
           "n_cells": info["n_cells"], "n_hanging": info["n_hanging"], "box_metric": info["box_metric"]}
    stream = torch.cuda.current_stream()
    for name, dt in (("vmult_fp32", torch.float32), ("vmult_fp64", torch.float64))[:2 if fp64 else 1]:
        x = torch.tensor(synthetic.uniform_vector(n, 71), device="cuda", dtype=dt)
        y = torch.empty_like(x)
        for _ in range(3):
            op.vmult(x, y)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(30)]
        for e0, e1 in evs:
            e0.record(stream)
            op.vmult(x, y)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in evs)
        byt = octree_bytes(n, info["n_cells"], k, 4 if dt == torch.float32 else 8,
                           box=bool(info["box_metric"]) and dt == torch.float32)
        out[name] = {"gdofs": n / (ms * 1e-3) / 1e9, "ms": ms,
                     "roofline": {"bound": "hbm", "achieved": byt / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                  "frac": byt / (ms * 1e-3) / 1e9 / hbm, "algorithmic_bytes": byt,
                                  "peak_kind": peak_kind}}
    return out


def sipg_measurement(mfx, synthetic, torch, np, dims=(128, 64, 64), k=4, solve=True):
    """The paper's multigrid benchmark discretisation: SIPG of degree 4 on the hyper-rectangle
    [0, 2] x [0, 1] x [0, 1] (128 x 64 x 64 cells, 65.5M DoFs, homogeneous Dirichlet data on every face).
    FP32 and FP64 vmult of the DG operator (device-resident vectors larger than L2), then PCG with the
    V-cycle of the DG -> continuous -> coarser hierarchy (Chebyshev(6) smoothing, exact coarse solve on
    2 x 1 x 1 cells as in the paper), FP64 and mixed (FP32 V-cycle inside FP64 defect correction), to 1e-10."""
    lengths = (2.0, 1.0, 1.0)
    verts = synthetic.lattice_vertices(*dims) * np.asarray(lengths)[None, :]
    mesh = mfx.Mesh.structured_box(*dims, verts)
    op = mfx.Operator(mesh, k, discretization=mfx.SIPG)
    n = op.n_dofs
    hbm, peak_kind = peaks()
    out = {"workload": "SIPG Q%d, %dx%dx%d cells of [0,2]x[0,1]x[0,1]" % ((k,) + tuple(dims)), "n_dofs": n}
    stream = torch.cuda.current_stream()
    for name, dt, nbytes in (("vmult_fp32", torch.float32, 8), ("vmult_fp64", torch.float64, 16)):
        x = torch.tensor(synthetic.uniform_vector(n, 61), device="cuda", dtype=dt)
        y = torch.empty_like(x)
        for _ in range(3):
            op.vmult(x, y)
        reps = 30 if dt == torch.float32 else 8
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            op.vmult(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = nbytes * n / (ms * 1e-3) / 1e9
        out[name] = {"gdofs": n / (ms * 1e-3) / 1e9, "ms": ms, "algorithmic_bytes": nbytes * n,
                     "achieved_gbs": gbs, "hbm_frac": gbs / hbm, "peak_kind": peak_kind}
        del x, y
    del op
    if not solve:
        return out
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = mfx.Multigrid(mesh, k, smoother_degree=6, discretization=mfx.SIPG)
    torch.cuda.synchronize()
    out["mg_levels"] = g.n_levels
    out["mg_setup_seconds"] = time.perf_counter() - t0
    b = torch.tensor(synthetic.gaussian_vector(n, 62), device="cuda")
    for name, mixed in (("mg_fp64", False), ("mg_mixed", True)):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.solve(b, x, tol=1e-10, mixed=mixed, inner_tol=1e-4)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "status": st["status"], "iterations": st["iterations"],
                     "inner_iterations": st["inner_iterations"], "rel_residual": st["rel_residual"]}
        if not mixed:
            # residual reduction per MG-preconditioned CG iteration
            out[name]["convergence_rate"] = st["rel_residual"] ** (1.0 / max(1, st["iterations"]))
    return out


if __name__ == "__main__":
    main()
