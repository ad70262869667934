"""Particle merging on the CUDA path (pic_merge) against the oracle's
(tests/test_oracle_merge.py pins it): the same pairs, ids and merged states
in FP64 (1e-12), a step after the merge, the mixed path's conservation, and
a cell too full for one block."""
import numpy as np
import pytest

import parity as P
import workloads as W
from oracle import C_BIRTHS, Oracle

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


def by_id(p):
    o = np.argsort(p["id"], kind="stable")
    return {k: np.asarray(v)[o] for k, v in p.items()}


def nerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if a.size == 0:
        return 0.0
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a).max())


def _cfg(prec):
    cfg = W.config("c1", precision=prec)
    for sp in cfg["species"]:
        sp["n_init"] = 0
        sp["capacity"] = 400_000
    return cfg


def _pair(pic, cfg, seed=3):
    e = W.random_particles(cfg, 0, 60_000, seed=seed, hot=3.0, accel=2e14, wscale=1.5e6)
    i = W.random_particles(cfg, 1, 40_000, seed=seed + 1, hot=30.0, accel=5e9, wscale=1.5e6)
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    for s, p in ((0, e), (1, i)):
        pic.pic_set_particles(h, s, p)
        o.set_particles(s, p)
    return h, o


DV = {0: 1.5e6, 1: 2e4}


def test_merge_matches_the_oracle_fp64_and_a_step_after_it(pic):
    cfg = _cfg("fp64")
    h, o = _pair(pic, cfg)
    for s in (0, 1):
        n_g, e_g = pic.pic_merge(h, s, 0.5, DV[s])
        n_o, e_o = o.merge(s, 0.5, DV[s])
        assert n_g == n_o and n_o > 500, (s, n_g, n_o)
        assert abs(e_g - e_o) <= 1e-9 * abs(e_o), (s, e_g, e_o)
        g, ref = by_id(pic.pic_get_particles(h, s)), by_id(o.get_particles(s))
        assert np.array_equal(g["id"], ref["id"])
        # element by element (tests/parity.py; no field yet: accelerations relative to themselves)
        e = P.errors(cfg, s, g, ref, 0.0, P.w_ref_table(cfg, s))
        assert e.max() <= 1e-12, (s, float(e.max()))
    # the deposit was redone: rho and chi as the oracle deposits them
    o.deposit()
    o.finalize()
    f = pic.pic_get_fields(h)
    for name in ("rho", "chi"):
        assert nerr(f[name], o.grid(name)) < 1e-12, name
    pic.pic_set_step(h, 17)
    o.set_step(17)
    assert pic.pic_step(h, 1) == 0
    o.step(1)
    f = pic.pic_get_fields(h)
    assert nerr(f["phi"], o.grid("phi")) < 1e-12
    emax = P.e_max({k: o.grid(k) for k in ("Ez", "Er")})
    for s in (0, 1):
        g, ref = by_id(pic.pic_get_particles(h, s)), by_id(o.get_particles(s))
        assert np.array_equal(g["id"], ref["id"])
        e = P.errors(cfg, s, g, ref, emax, P.w_ref_table(cfg, s))
        assert e.max() <= 1e-12, (s, float(e.max()))
    assert list(pic.pic_moments(h)["counters"][C_BIRTHS:C_BIRTHS + 2]) == list(o.counters()[0][C_BIRTHS:C_BIRTHS + 2])


def test_mixed_merge_keeps_charge_and_momentum(pic):
    cfg = _cfg("mixed")
    h, o = _pair(pic, cfg, seed=9)
    for s in (0, 1):
        before = pic.pic_get_particles(h, s)
        n_g, e_g = pic.pic_merge(h, s, 0.5, DV[s])
        n_o, _ = o.merge(s, 0.5, DV[s])
        assert abs(n_g - n_o) <= max(20, 0.01 * n_o), (s, n_g, n_o)
        after = pic.pic_get_particles(h, s)
        assert len(after["id"]) == len(before["id"]) - n_g
        w0, w1 = before["w"], after["w"]
        assert abs(w1.sum() - w0.sum()) <= 1e-6 * w0.sum()
        for k in ("vr", "vz"):
            p0, p1 = (w0 * before[k]).sum(), (w1 * after[k]).sum()
            assert abs(p1 - p0) <= 1e-5 * np.abs(w0 * before[k]).sum(), (s, k)
    assert pic.pic_step(h, 2) == 0


def test_a_cell_too_full_is_reported_and_left_alone(pic):
    cfg = _cfg("fp64")
    n = 1200
    rng = np.random.default_rng(2)
    dz, dr = cfg["L"] / (cfg["nz"] - 1), cfg["R"] / (cfg["nr"] - 1)
    zero = np.zeros(n)
    p = dict(z=(5 + rng.uniform(0, 1, n)) * dz, r=(20 + rng.uniform(0, 1, n)) * dr, vr=rng.normal(0, 1e3, n),
             vt=rng.normal(0, 1e3, n), vz=rng.normal(0, 1e3, n), ar=zero, az=zero, w=np.full(n, 10.0),
             id=np.arange(n, dtype=np.uint64))
    h = pic.pic_init(cfg, load=False)
    pic.pic_set_particles(h, 0, p)
    with pytest.raises(pic.PicError) as err:
        pic.pic_merge(h, 0, 0.5, 1e9)
    assert err.value.status == pic.PIC_ERR_CAPACITY
    assert pic.pic_get_counts(h)["n_alive"][0] == n


def test_merge_with_the_xyz_pusher_and_held_ions(pic):
    """a_theta merges like v_theta (X-Y-Z pusher); ions merged while a
    subcycled run holds them, then two steps (a holding and a moving pass):
    the same as the oracle in FP64."""
    cfg = dict(_cfg("fp64"), pusher="xyz", ion_subcycle=2, split_every=0)
    rng = np.random.default_rng(12)
    e = W.random_particles(cfg, 0, 30_000, seed=21, hot=3.0, accel=2e14, wscale=1.5e6)
    i = W.random_particles(cfg, 1, 30_000, seed=22, hot=30.0, accel=5e9, wscale=1.5e6)
    e["at"] = rng.normal(0.0, 2e14, 30_000)
    i["at"] = rng.normal(0.0, 5e9, 30_000)
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    for s, p in ((0, e), (1, i)):
        pic.pic_set_particles(h, s, p)
        o.set_particles(s, p)
        o.set_at(s, p["at"])
    pic.pic_set_step(h, 0)
    o.set_step(0)
    assert pic.pic_step(h, 1) == 0  # pass 0 holds the ions; newborn ions wait in their births
    o.step(1)
    for s in (0, 1):
        n_g, _ = pic.pic_merge(h, s, 0.5, DV[s])
        n_o, _ = o.merge(s, 0.5, DV[s])
        assert n_g == n_o and n_o > 100, (s, n_g, n_o)
    assert pic.pic_step(h, 2) == 0
    o.step(2)
    for s in (0, 1):
        g = by_id(pic.pic_get_particles(h, s))
        ref = o.get_particles(s)
        ref["at"] = o.get_at(s)
        ref = by_id(ref)
        assert np.array_equal(g["id"], ref["id"])
        for k in FIELDS + ("at",):
            assert nerr(g[k], ref[k]) <= 1e-11, (s, k, nerr(g[k], ref[k]))
