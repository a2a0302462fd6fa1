"""The N > 1 path of bench.py on CPU: two gloo ranks.

Each rank labels its own lattice (replicas, no data-path collective); the step
time is the maximum over ranks and the job throughput counts every rank's
sites.  The reference arm runs on rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(ms[rank], dist, device="cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_max_over_two_gloo_ranks():
    world = 2
    ms = [3.25, 7.5]
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), ms, out), nprocs=world, join=True)
    assert out[0] == max(ms) and out[1] == max(ms)
    # whole-job throughput: both ranks' sites in the slowest rank's time
    assert bench.job_gsites_per_s(world, 1024 ** 3, max(ms)) == pytest.approx(2 * 1024 ** 3 / 7.5e-3 / 1e9)


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(4.0) == 4.0
    assert bench.job_gsites_per_s(1, 1000, 1.0) == pytest.approx(1e-3)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(Args, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys):
    """The reference arm's JSON line: the oracle timed on the host on a bounded sample,
    with the metric, unit and direction of the GPU arm and its own cpu_baseline and e2e."""
    import json

    class Args:
        steps, warmup, gpus = 1, 0, 1
    bench.run_reference(Args, rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "Gsites/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "Gsites/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["steps"] == 1 and line["n_gpus"] == 1
