"""Multi-process host logic of the replica path (world size 2, gloo, CPU).

With N > 1 every rank runs its own replica of the step on its own GPU and
no data moves between ranks; the only cross-rank steps are the barriers
around the timed region and the maximum of the per-rank times.  These
tests run that host logic as two gloo ranks on the CPU, and check that the
reference arm's non-zero ranks leave without work.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, per_rank_ms, units, out):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        mx = bench.max_over_ranks(per_rank_ms[rank], world, "cpu")
        value = bench.whole_job_rate(units, world, mx[0])
        dist.barrier()
        out.put((rank, mx, value))
    finally:
        dist.destroy_process_group()


def _run_ranks(per_rank_ms, units):
    world = len(per_rank_ms)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, per_rank_ms, units, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return dict((r, (mx, v)) for r, mx, v in res)


def test_max_over_ranks_gloo_world2():
    # rank 1 is the slow one for the device time, rank 0 for the end-to-end time
    per_rank = [[10.0, 31.5], [14.25, 20.0]]
    units = 20_000_000
    res = _run_ranks(per_rank, units)
    for r in (0, 1):
        mx, value = res[r]
        assert mx == [14.25, 31.5]
        # whole-job rate: both ranks' units over the slowest rank's time
        assert value == pytest.approx(2 * units / 14.25e-3, rel=1e-12)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks([3.0, 4.5], 1) == [3.0, 4.5]
    assert bench.whole_job_rate(1000, 1, 2.0) == pytest.approx(500_000.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
