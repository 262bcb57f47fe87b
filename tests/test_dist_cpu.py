"""The multi-GPU host path of bench.py (replicas, barrier, max over ranks, whole-job value) on
two CPU processes with the gloo backend."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(backend="gloo")
    bench.barrier(w)
    ms = 10.0 * (r + 1)                                # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, w)
    value = bench.job_throughput(256 ** 3, 100, w, ms_max)
    out.put((r, w, ms_max, value))
    dist.destroy_process_group()


def test_two_rank_replicas_report_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for _, w, ms_max, value in res:
        assert w == 2 and ms_max == 20.0
        # both replicas' points, timed by the slower rank
        assert value == pytest.approx(2 * 256 ** 3 * 100 / 0.020)
