"""The multi-rank path of bench.py on CPU (gloo, world size 2): the whole-job
rate adds every rank's units and divides by the slowest rank's time, and the
reference arm runs on rank 0 only.  The data path itself has no collective
(each rank runs an independent replica), so this is the only exchange."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, units, seconds, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        rate, t = bench.whole_job_rate(units[rank], seconds[rank], world, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    q.put((rank, rate, t))


@pytest.mark.parametrize("units,seconds", [((100, 300), (2.0, 4.0)), ((7, 7), (1.5, 0.5))])
def test_two_gloo_ranks_add_units_and_take_the_slowest_time(units, seconds):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, units, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            rank, rate, t = q.get(timeout=120)
            got[rank] = (rate, t)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    want = (sum(units) / max(seconds), max(seconds))
    assert got[0] == pytest.approx(want) and got[1] == pytest.approx(want)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.whole_job_rate(10, 2.0, 1) == (5.0, 2.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    import bench
    bench.run_reference(argparse.Namespace(steps=1, warmup=3), rank=1, world=2)
    assert capsys.readouterr().out == ""
