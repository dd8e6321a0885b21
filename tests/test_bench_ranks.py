"""Multi-rank (replica) aggregation of bench.py, on CPU with the gloo backend and two ranks:
the job time is the slowest rank's and the throughput counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, rate = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000.0, dist, "cpu")
    out[rank] = (t, rate)
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_aggregation_takes_slowest_rank_and_total_work():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    for rank in (0, 1):
        t, rate = out[rank]
        assert t == 15.0
        assert abs(rate - 2 * 1000.0 / 15e-3) < 1e-6


def test_single_process_aggregation():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    t, rate = bench.aggregate_ranks(20.0, 500.0)
    assert t == 20.0 and abs(rate - 500.0 / 20e-3) < 1e-9


def test_oracle_baseline_times_exactly_the_requested_steps():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.cpu_baseline(sub=3, steps=4, warmup=1, one_core=False)
    assert cb["kind"] == "oracle" and cb["unit"] == "GDoF/s" and cb["cores"] >= 1
    assert "4 SpMVs" in cb["sample"] and cb["value"] > 0 and cb["ms_per_spmv"] > 0


def test_reference_arm_line(monkeypatch, capsys):
    """The reference arm prints one JSON line with the main arm's metric, unit, direction and workload,
    and its own e2e and cpu_baseline objects; ranks other than 0 print nothing."""
    import argparse
    import json
    import sys
    sys.path.insert(0, ROOT)
    import bench
    fake = {"value": 0.02, "unit": "GDoF/s", "cores": 4, "kind": "oracle", "ms_per_spmv": 6.0,
            "one_core_value": None, "sample": "test"}
    monkeypatch.setattr(bench, "cpu_baseline", lambda **kw: dict(fake, steps=kw["steps"]))
    args = argparse.Namespace(gpus=1, steps=7, warmup=3)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GDoF/s"
    assert line["higher_is_better"] is True and line["config"]["workload"] == bench.WORKLOAD
    assert line["steps"] == 7 and line["warmup"] == 3 and line["ms_per_step"] == 6.0
    assert line["cpu_baseline"]["steps"] == 7 and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": 0.02, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def test_clock_record_rejection_rule():
    """Slowdown reasons or SM clocks well below their maximum with no reason reject a timed region (it is
    measured once more); a power cap alone does not."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9}
    assert not bench.clocks_rejected(ok) and not bench.clocks_rejected(None)
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1600.0, reasons=["sw_power_cap"]))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))
