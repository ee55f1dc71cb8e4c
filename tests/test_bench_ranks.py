"""The replica path of bench.py on CPU (gloo, world size 2): each rank times its
own block; the job's time per step is the slowest rank's and its rate counts the
solves of all ranks.  The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [4.0 + rank, 5.0 + 2 * rank]               # rank 1 is the slower one
    got_ms, got_val = bench.aggregate_ranks(ms, world, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got_ms, got_val))


def test_max_over_ranks_and_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val in res:
        assert ms == [5.0, 7.0]                      # the slowest rank's times on every rank
        assert val == pytest.approx([2 * 1000.0 / 5.0, 2 * 1000.0 / 7.0])


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "hexagon_8x8_n256"
    bench.run_reference(A(), rank=1, world=2)       # returns at once, prints nothing
    assert capsys.readouterr().out == ""
