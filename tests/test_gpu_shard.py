"""One reactor's particles shared by two processes (Sec. 2.7) against the same
reactor in one process, FP64.

Two spawned processes on the one GPU, each a handle holding the particles of
one id parity, exchange their deposits through gloo on host copies after
every step (paper_1001_2969_gb300.shard); their kernels never wait on each
other.  Without births the shared run must be the one-process run: fields
to 1e-12, every particle element by element (tests/parity.py) with the same
ids, the collision, candidate and absorption counters summed over the
processes equal.  With ionisation and splitting, each process numbers its
newborns in its own residue class: after the first step the fields still
agree, the parents agree, the newborn states agree as a set and every id is
unique across the processes.
"""
import os
import socket
import sys

import numpy as np
import pytest

import parity as P
import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ("r", "z", "vr", "vt", "vz", "ar", "az", "w")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _cfg(births):
    cfg = W.scaled(W.config("c1", precision="fp64"), 20_000)
    if not births:
        # electrons: elastic and excitation only (no ionisation), no split
        xs = dict(cfg["xsec"][0])
        keep = [k for k, kind in enumerate(xs["kind"]) if kind != "ionize"]
        xs["sigma"] = np.asarray(xs["sigma"])[keep]
        xs["threshold"] = np.asarray(xs["threshold"])[keep]
        xs["kind"] = [xs["kind"][k] for k in keep]
        cfg["xsec"] = [xs, cfg["xsec"][1]]
        cfg["split_every"] = 0
    else:
        cfg["split_every"] = 1
        # room for the split copies (up to 3 per particle, see _reference)
        cfg["species"] = [dict(sp, capacity=120_000) for sp in cfg["species"]]
    return cfg


def _worker(rank, world, port, births, parts, steps, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1001_2969_gb300 import build, pic, shard

    build()
    cfg = _cfg(births)
    h = pic.pic_init(cfg, load=False)
    first_free = []
    for s in (0, 1):
        p = parts[s]
        mine = (p["id"] % world) == rank
        pic.pic_set_particles(h, s, {k: np.asarray(v)[mine] for k, v in p.items()})
        first_free.append(int(p["id"].max()) + 1)
    shard.number_newborns(h, rank, world, first_free)
    shard.exchange_deposit(h)  # the load's deposit, summed, before the first solve
    st = shard.step(h, steps)
    out = dict(status=st, fields=pic.pic_get_fields(h),
               particles=[pic.pic_get_particles(h, s) for s in (0, 1)],
               counters=pic.pic_moments(h)["counters"])
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def _run_shared(births, parts, steps):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, births, parts, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r, out = q.get(timeout=600)
        got[r] = out
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return got


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic as Pm

    build()
    return Pm


def _reference(pic, births, steps):
    cfg = _cfg(births)
    loaded = pic.pic_init(cfg)
    parts = [pic.pic_get_particles(loaded, s) for s in (0, 1)]
    parts = [{k: np.asarray(p[k]) for k in FIELDS + ("id",)} for p in parts]
    pic.pic_destroy(loaded)
    if births:
        # heavier particles than the split's reference weight: every step splits
        for p in parts:
            p["w"] = p["w"] * (1.0 + 3.0 * ((p["id"] % 7).astype(np.float64) / 7.0))
    h = pic.pic_init(cfg, load=False)
    for s in (0, 1):
        pic.pic_set_particles(h, s, parts[s])
    assert pic.pic_step(h, steps) == 0
    ref = dict(fields=pic.pic_get_fields(h), particles=[pic.pic_get_particles(h, s) for s in (0, 1)],
               counters=pic.pic_moments(h)["counters"])
    return cfg, parts, ref


def _union(got, s):
    a, b = got[0]["particles"][s], got[1]["particles"][s]
    return {k: np.concatenate([np.asarray(a[k]), np.asarray(b[k])]) for k in FIELDS + ("id",)}


def test_shared_reactor_matches_one_process_without_births(pic):
    steps = 3
    cfg, parts, ref = _reference(pic, False, steps)
    got = _run_shared(False, parts, steps)
    for r in (0, 1):
        assert got[r]["status"] == 0
        for k in ("phi", "Ez", "Er"):
            o = ref["fields"][k]
            assert np.abs(got[r]["fields"][k] - o).max() <= 1e-12 * np.abs(o).max(), (r, k)
    grids = {k: ref["fields"][k] for k in ("Ez", "Er")}
    for s in (0, 1):
        g, o = P.by_id(_union(got, s)), P.by_id(ref["particles"][s])
        assert np.array_equal(g["id"], o["id"])
        e = P.errors(cfg, s, g, o, P.e_max(grids), P.w_ref_table(cfg, s))
        assert e.max() <= 1e-12, (s, float(e.max()))
    idx = list(range(0, 10)) + list(range(16, 22))  # collisions, candidates, absorptions
    csum = got[0]["counters"] + got[1]["counters"]
    assert [int(csum[k]) for k in idx] == [int(ref["counters"][k]) for k in idx]
    assert ref["counters"][0] > 0 and ref["counters"][4] > 0  # collisions happened


def test_shared_reactor_with_births_keeps_ids_unique(pic):
    cfg, parts, ref = _reference(pic, True, 1)
    got = _run_shared(True, parts, 1)
    for r in (0, 1):
        assert got[r]["status"] == 0
        o = ref["fields"]["phi"]
        assert np.abs(got[r]["fields"]["phi"] - o).max() <= 1e-12 * np.abs(o).max()
    in_ids = [set(np.asarray(p["id"]).tolist()) for p in parts]
    grids = {k: ref["fields"][k] for k in ("Ez", "Er")}
    births = 0
    for s in (0, 1):
        g, o = P.by_id(_union(got, s)), P.by_id(ref["particles"][s])
        assert len(np.unique(g["id"])) == len(g["id"])  # unique across the processes
        assert len(g["id"]) == len(o["id"])
        gp = np.array([i in in_ids[s] for i in g["id"].tolist()])
        op = np.array([i in in_ids[s] for i in o["id"].tolist()])
        assert np.array_equal(g["id"][gp], o["id"][op])  # the parents, by id
        e = P.errors(cfg, s, {k: g[k][gp] for k in FIELDS}, {k: o[k][op] for k in FIELDS},
                     P.e_max(grids), P.w_ref_table(cfg, s))
        assert e.max() <= 1e-12
        # newborns: the same states as a set (their ids differ)
        gn = {k: g[k][~gp] for k in FIELDS}
        on = {k: o[k][~op] for k in FIELDS}
        births += len(gn["r"])
        go, oo = np.lexsort((gn["z"], gn["r"])), np.lexsort((on["z"], on["r"]))
        e = P.errors(cfg, s, {k: gn[k][go] for k in FIELDS}, {k: on[k][oo] for k in FIELDS},
                     P.e_max(grids), P.w_ref_table(cfg, s))
        assert e.max(initial=0.0) <= 1e-12
    assert births > 100
