"""The multi-rank path of bench.py on CPU: two gloo ranks (world_size 2).

Every rank runs its own batch (replicas, weak scaling); the job time is the
slowest rank's, and only rank 0 prints.  The reference arm does no work on
ranks other than 0.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 * (rank + 1)                 # rank 1 is the slow one
    got = bench.max_over_ranks(local_ms, dist)
    value = bench.weak_scaling_value(8, 4, world, got)
    out.put((rank, got, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == 20.0
        # 2 directions x 8 right-hand sides x 4 steps x 2 ranks in 20 ms
        assert value == pytest.approx(2 * 8 * 4 * 2 / 0.020)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_scaling_value(8, 10, 1, 1000.0) == pytest.approx(160.0)


def test_reference_arm_skips_other_ranks(capsys):
    import argparse

    import bench
    import synth
    args = argparse.Namespace(steps=1, warmup=0, ref_seconds=1.0, gpus=2)
    bench.reference_arm(args, "2d_1024_m16_b8", rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_matches_the_gpu_arm_config(capsys):
    """Rank 0 times the compiled oracle for real steps and prints the contract's line
    with the same config block the GPU arm prints for that workload."""
    import argparse
    import json

    import bench
    import synth
    args = argparse.Namespace(steps=2, warmup=0, ref_seconds=1.0, gpus=1)
    bench.reference_arm(args, "1d_n1024_m8_b1", rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["value"] > 0
    assert line["config"] == bench.headline_config(synth.workload("1d_n1024_m8_b1"), 1)
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["cpu_model"]
    # each step is one forward and one adjoint apply: value = 2 steps x 2 applies / total time
    assert line["value"] == __import__("pytest").approx(2 * 2 / (2 * line["ms_per_step"] / 1000.0))
    assert line["e2e"] == {"value": line["value"], "unit": "applies/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
