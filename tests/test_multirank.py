"""The N > 1 path of bench.py on CPU: two gloo ranks, each an independent
reactor replica, combine into whole-job figures (the particle-steps of all
ranks over the slowest rank's time)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, root, q):
    import torch.distributed as dist

    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = (12.0, 15.0)[rank]         # device-timed region of this rank
    psteps = (1.0e6, 2.5e6)[rank]   # particle-steps this rank processed
    e2e_s = (0.50, 0.40)[rank]
    e2e_n = (3.0e5, 4.0e5)[rank]
    q.put((rank, bench.whole_job(ms, psteps, e2e_s, e2e_n, world, device="cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, root, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest time and the summed work
    for r in (0, 1):
        assert got[r] == (15.0, 3.5e6, 0.50, 7.0e5)
    value = got[0][1] / (got[0][0] * 1e-3)
    assert value == pytest.approx(3.5e6 / 15e-3)


def test_one_rank_is_its_own_whole_job():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    assert bench.whole_job(3.0, 10.0, 0.5, 4.0, 1) == (3.0, 10.0, 0.5, 4.0)
