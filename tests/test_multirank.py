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


def _shard_worker(rank, world, port, root, q):
    """The deposit exchange of a shared reactor on a fake handle (no GPU)."""
    import numpy as np
    import torch.distributed as dist

    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1001_2969_gb300 import pic, shard

    class Fake:
        nz, nr = 3, 4

    h = Fake()
    state = {"Ne": np.full((3, 4), 1.0 + rank), "Ni": np.arange(12.0).reshape(3, 4) * (rank + 1),
             "q": np.array([1.0, 2.0, 3.0]) * (10 ** rank), "steps": 0}
    pic.pic_get_deposit = lambda hh: {k: state[k].copy() for k in ("Ne", "Ni", "q")}

    def setd(hh, Ne, Ni, q=None):
        state["Ne"], state["Ni"], state["q"] = (np.asarray(Ne).reshape(3, 4), np.asarray(Ni).reshape(3, 4),
                                                np.asarray(q))

    def stepf(hh, n):
        state["steps"] += n
        return pic.PIC_OK

    pic.pic_set_deposit = setd
    pic.pic_step = stepf
    st = shard.step(h, 2, None)
    q.put((rank, st, state["steps"], state["Ne"].tolist(), state["Ni"].tolist(), state["q"].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_shared_reactor_deposit_exchange_over_two_gloo_ranks():
    """Each rank's deposit (electrons, ions, wall charges) is replaced by the sum
    over the ranks after every step (Sec. 2.7's all-reduce before the solve)."""
    import numpy as np
    import torch.multiprocessing as mp

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, root, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r, *rest = q.get(timeout=180)
        got[r] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # two steps: the first exchange sums (1 + 2), the second sums the sums
    for r in (0, 1):
        st, steps, Ne, Ni, qq = got[r]
        assert st == 0 and steps == 2
        np.testing.assert_array_equal(np.array(Ne), np.full((3, 4), 2.0 * 3.0))
        np.testing.assert_array_equal(np.array(Ni), 2.0 * 3.0 * np.arange(12.0).reshape(3, 4))
        np.testing.assert_array_equal(np.array(qq), 2.0 * 11.0 * np.array([1.0, 2.0, 3.0]))
