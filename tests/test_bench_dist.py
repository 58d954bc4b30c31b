"""The multi-replica path of bench.py on CPU: two gloo ranks (127.0.0.1) aggregate their timings
the way the GPU ranks do - the slowest rank's time, all ranks' updates."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms_local = 100.0 + 50.0 * rank              # rank 1 is the slow one
    ms_max, value = bench._job_throughput(ms_local, 1.0e9, world, device="cpu")
    e2e = bench._job_e2e(2.0e9 / (1 + rank), world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms_max, value, e2e))


def test_two_replicas_report_the_slowest_rank_and_the_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, e2e in res:
        assert ms_max == 150.0                        # max over ranks
        assert abs(value - 2 * 1.0e9 / 0.150) < 1e-3  # all ranks' updates / slowest time
        assert abs(e2e - 2 * 1.0e9) < 1e-3            # slowest rank's rate x ranks
