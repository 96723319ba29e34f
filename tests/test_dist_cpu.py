"""The multi-process path of bench.py (replicas: barrier, max over ranks) with two gloo ranks
on the CPU.  The solver path itself does not shard; ranks only agree on the timing."""
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

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.dist_env()
        assert (w, r, l) == (world, rank, rank)
        bench.barrier(world)
        out[rank] = bench.max_over_ranks(10.0 + rank, world)
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert dict(out) == {0: 11.0, 1: 11.0}


def test_single_rank_helpers_need_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)


def _reference_worker(rank, world, port, out):
    # bench.py --impl reference under two gloo ranks, on a 4^4 lattice with short oracle samples
    import contextlib
    import io
    import types

    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    bench.DIMS = (4, 4, 4, 4)
    sample = bench.oracle_sample
    bench.oracle_sample = lambda seconds, iters: sample(0.05, iters)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    buf = io.StringIO()
    try:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(types.SimpleNamespace(gpus=world, steps=2, warmup=1), world, rank)
    finally:
        dist.destroy_process_group()
    out[rank] = buf.getvalue()


def test_reference_arm_prints_one_line_on_rank_zero_only():
    import json
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_reference_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[1] == ""
    lines = out[0].strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "ms" and line["higher_is_better"] is False
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"] and "sample" in line["cpu_baseline"]
    assert line["e2e"] == {"value": line["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["iterations"] > 0 and line["true_residual"] <= 1e-10
