"""bench.py's multi-rank bookkeeping (weak scaling over independent maps),
run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx = bench.max_over_ranks(100.0 + 50.0 * rank, dist, torch.device("cpu"))
    out[rank] = (mx, bench.aggregate_value(world, 3, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_value():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        mx, val = out[r]
        assert mx == 150.0
        assert val == pytest.approx(2 * 3 / 0.150)


def test_single_rank_defaults():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.aggregate_value(1, 2, 4000.0) == pytest.approx(0.5)


def test_analysis_traffic_only_for_the_captured_variant(monkeypatch):
    import bench
    if bench.ANALYSIS_DRAM_FULL_BAND["bytes"] is None:  # no capture of the current kernel
        assert bench.analysis_traffic(1024, 22.0, 1) is None
    ref = dict(bench.ANALYSIS_DRAM_FULL_BAND, bytes=2.0e8)
    monkeypatch.setattr(bench, "ANALYSIS_DRAM_FULL_BAND", ref)
    tuning = {"ana_np": [4, ref["variant"]["ana_np"]], "ana_queue": ref["variant"]["ana_queue"],
              "ana_packed": ref["variant"]["ana_packed"],
              "ana_global_acc": ref["variant"]["ana_global_acc"]}
    v = bench.analysis_variant(tuning)
    assert v == ref["variant"]
    # a launch covering the full band's terms carries the captured bytes
    gflop = 7.0 * ref["terms"] / 1e9
    assert bench.analysis_traffic(ref["nside"], gflop, 1, v) == pytest.approx(ref["bytes"])
    assert bench.analysis_traffic(ref["nside"], 2 * gflop, 4, v) == pytest.approx(ref["bytes"] / 2)
    other = dict(v, ana_queue=1, ana_packed=0)
    assert bench.analysis_traffic(ref["nside"], gflop, 1, other) is None
    assert bench.analysis_traffic(ref["nside"] // 2, gflop, 1, v) is None
    assert bench.analysis_traffic(ref["nside"], gflop, 0, v) is None


def test_reference_arm_times_each_step(osht):
    """The reference arm (the oracle on the host cores) times every step as
    its own bounded sample and prints the contract's keys; other ranks do
    no work."""
    import argparse
    import bench
    args = argparse.Namespace(nside=8, steps=3, warmup=1, cpu_sample_s=0.3)
    out = bench.run_reference(args, 0, 1)
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert k in out
    assert out["impl"] == "reference" and out["value"] > 0
    assert out["ms_per_step"] == pytest.approx(1e3 * 3 / out["value"] / 3)
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0
    assert bench.run_reference(args, 1, 2) is None
