"""Parity at the full bench workload (c2: 129 x 513 nodes, 1e7 + 1e7 particles), in the
launch configuration bench.py times.

The oracle runs the same load and one full step in FP64 (C, single thread, ~10 s);
sampled particles, the whole potential and the conservation laws are compared.
"""
import numpy as np
import pytest

import parity as P
import workloads as W
from oracle import C_ABS, C_BIRTHS, Oracle

pytestmark = pytest.mark.gpu

FIELDS = ("r", "z", "vr", "vt", "vz", "ar", "az", "w")


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic as P

    build()
    return P


@pytest.fixture(scope="module")
def oracle_c2():
    """The oracle's c2 load and its first step (shared by the tests of this module)."""
    cfg = W.config("c2")
    o = Oracle(cfg)
    o.load()
    loaded = [o.get_particles(s) for s in (0, 1)]
    q = [sp["q"] for sp in cfg["species"]]
    charge0 = sum(q[s] * loaded[s]["w"].sum() for s in (0, 1))
    o.step(1)
    o.finalize()
    after = [o.get_particles(s) for s in (0, 1)]
    counters = o.counters()
    grids = {k: o.grid(k) for k in ("phi", "Ez", "Er", "rho", "chi")}
    V = o.node_volumes()
    return dict(cfg=cfg, loaded=loaded, after=after, counters=counters, grids=grids, V=V,
                charge0=charge0)


def _index(p):
    o = np.argsort(p["id"], kind="stable")
    return {k: np.asarray(v)[o] for k, v in p.items()}


def _sample_ids(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False)).astype(np.uint64)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_full_size_load_and_first_step(pic, oracle_c2, prec):
    ref = oracle_c2
    cfg = W.config("c2", precision=prec)
    h = pic.pic_init(cfg)
    # the load: sampled particles and exact cells
    for s in (0, 1):
        g = _index(pic.pic_get_particles(h, s))
        o = _index(ref["loaded"][s])
        assert np.array_equal(g["id"], o["id"])
        ids = _sample_ids(len(o["id"]), 2000, seed=10 + s)
        tol = 1e-12 if prec == "fp64" else 2e-7
        e = P.errors(cfg, s, {k: g[k][ids] for k in FIELDS}, {k: o[k][ids] for k in FIELDS}, 0.0,
                     P.w_ref_table(cfg, s))
        assert e.max() <= tol, float(e.max())
        dz, dr = cfg["L"] / (cfg["nz"] - 1), cfg["R"] / (cfg["nr"] - 1)
        i = np.floor(o["z"][ids] / dz).astype(np.int64)
        j = np.floor(o["r"][ids] / dr).astype(np.int64)
        assert np.array_equal(g["cell"][ids], j * (cfg["nz"] - 1) + i)
    # one step, as bench.py runs it
    assert pic.pic_step(h, 1) == pic.PIC_OK
    f = pic.pic_get_fields(h)
    phi_tol = 1e-12 if prec == "fp64" else 1e-6
    for name in ("phi", "Ez", "Er"):
        o = ref["grids"][name]
        assert np.abs(f[name] - o).max() <= phi_tol * np.abs(o).max(), name
    m = pic.pic_moments(h)
    oc, oq = ref["counters"]
    q = [sp["q"] for sp in cfg["species"]]
    Qs = abs(q[0]) * ref["loaded"][0]["w"].sum()  # charge of one species
    tolQ = 1e-12 if prec == "fp64" else 1e-6
    charge1 = 0.0
    for s in (0, 1):
        g_raw = pic.pic_get_particles(h, s)
        g = _index(g_raw)
        # particle-count conservation holds exactly on both sides
        absorbed = m["counters"][C_ABS + 3 * s: C_ABS + 3 * s + 3].sum()
        n0 = cfg["species"][s]["n_init"]
        assert len(g["id"]) == n0 - absorbed + m["counters"][C_BIRTHS + s]
        charge1 += q[s] * g["w"].sum()
        if prec == "fp64":
            assert list(m["counters"][:22]) == list(oc[:22])
        # every particle once, in cell order; sampled particles element by
        # element (FP64: same ids and cells; mixed: each outlier explained by
        # FP32 rounding at a decision threshold)
        P.compare_species(cfg, s, g_raw, ref["after"][s], prec, inputs=ref["loaded"][s],
                          grids=ref["grids"], step=0, sample=5000, seed=20 + s)
    # charge: what is inside plus what the walls took is conserved (ionisation makes pairs)
    assert abs(charge1 + m["charge"].sum() - ref["charge0"]) <= tolQ * Qs
    # deposit: the node sums add up to the charge the particles hold
    deposited = (f["rho"] * ref["V"]).sum()
    assert abs(deposited - charge1) <= tolQ * Qs
