"""Batched reactors and the particle-pass shapes.

A batch steps independent reactors of uneven mesh and particle count as one
CUDA graph per step (one branch per reactor); each reactor must come out as
if stepped alone.  Every particle-pass shape must give the default shape's
results, and the tuner must pick valid shapes.
"""
import numpy as np
import pytest

import parity as P
import workloads as W
from oracle import Oracle

pytestmark = pytest.mark.gpu

FIELDS = ("r", "z", "vr", "vt", "vz", "w")


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
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a).max())


def same_state(pic, ha, hb, tol, exact_ids):
    fa, fb = pic.pic_get_fields(ha), pic.pic_get_fields(hb)
    for k in ("phi", "rho", "chi", "Ez"):
        assert nerr(fa[k], fb[k]) < tol, k
    ca, cb = pic.pic_get_counts(ha), pic.pic_get_counts(hb)
    assert ca["step"] == cb["step"]
    for s in (0, 1):
        a, b = by_id(pic.pic_get_particles(ha, s)), by_id(pic.pic_get_particles(hb, s))
        if exact_ids:
            assert np.array_equal(a["id"], b["id"])
            for k in FIELDS:
                assert nerr(a[k], b[k]) < 100 * tol, k
        else:
            common = np.intersect1d(a["id"], b["id"])
            assert len(common) >= len(a["id"]) - 5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_reactors_stepped_alone(pic, prec):
    cfgs = W.batch_configs(n=5, seed=7, n_lo=5_000, n_hi=40_000, precision=prec)
    alone = [pic.pic_init(c) for c in cfgs]
    batched = [pic.pic_init(c) for c in cfgs]
    b = pic.pic_batch_init(batched)
    # two calls: three steps then two (both buffer parities of every reactor)
    assert b.step(3) == [0] * len(cfgs)
    assert b.step(2) == [0] * len(cfgs)
    for h in alone:
        assert pic.pic_step(h, 5) == 0
    tol = 1e-11 if prec == "fp64" else 2e-5
    for ha, hb in zip(alone, batched):
        same_state(pic, ha, hb, tol, exact_ids=prec == "fp64")
        ma, mb = pic.pic_moments(ha), pic.pic_moments(hb)
        if prec == "fp64":
            assert list(ma["counters"][:22]) == list(mb["counters"][:22])
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_reactors_match_the_oracle(pic, prec):
    """Three reactors of an uneven draw (meshes, particle counts, pressures and
    voltages differ), stepped together, each against the oracle stepped
    alone: the first step element by element, two more steps (both buffer
    parities) in the fields, ids and counters."""
    cfgs = W.batch_configs(n=3, seed=11, n_lo=4_000, n_hi=30_000, precision=prec)
    meshes = {(c["nz"], c["nr"]) for c in cfgs}
    assert len(meshes) > 1
    hs = [pic.pic_init(c) for c in cfgs]
    b = pic.pic_batch_init(hs)
    oracles = []
    for c in cfgs:
        o = Oracle(c)
        o.load()
        oracles.append((o, [o.get_particles(s) for s in (0, 1)]))
    assert b.step(1) == [0] * len(cfgs)
    ftol = 1e-12 if prec == "fp64" else 1e-6
    for c, h, (o, loaded) in zip(cfgs, hs, oracles):
        o.step(1)
        grids = {k: o.grid(k) for k in ("phi", "Ez", "Er")}
        f = pic.pic_get_fields(h)
        for k in ("phi", "Ez", "Er"):
            assert nerr(f[k], grids[k]) < ftol, (c["name"], k)
        for s in (0, 1):
            P.compare_species(c, s, pic.pic_get_particles(h, s), o.get_particles(s), prec,
                              inputs=loaded[s], grids=grids, step=0)
        if prec == "fp64":
            oc, _ = o.counters()
            assert list(pic.pic_moments(h)["counters"][:22]) == list(oc[:22]), c["name"]
    assert b.step(2) == [0] * len(cfgs)
    for c, h, (o, _) in zip(cfgs, hs, oracles):
        o.step(2)
        f = pic.pic_get_fields(h)
        assert nerr(f["phi"], o.grid("phi")) < (1e-11 if prec == "fp64" else 1e-5), c["name"]
        if prec == "fp64":
            for s in (0, 1):
                assert np.array_equal(by_id(pic.pic_get_particles(h, s))["id"], by_id(o.get_particles(s))["id"])
            oc, _ = o.counters()
            assert list(pic.pic_moments(h)["counters"][:22]) == list(oc[:22]), c["name"]
    b.close()


def test_batch_reports_each_reactors_status(pic):
    cfgs = W.batch_configs(n=3, seed=3, n_lo=5_000, n_hi=20_000, precision="fp64")
    # reactor 1 cannot hold its births
    cfgs[1]["births_capacity"] = 1
    cfgs[1]["gas"] = dict(cfgs[1]["gas"], p_Pa=100.0)
    cfgs[1]["split_every"] = 1
    hs = [pic.pic_init(c) for c in cfgs]
    b = pic.pic_batch_init(hs)
    with pytest.raises(pic.PicError):
        b.step(2)
    b.close()
    # the others went on
    for k in (0, 2):
        assert pic.pic_get_counts(hs[k])["step"] == 2
    assert pic.pic_get_counts(hs[1])["step"] < 2


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_particle_pass_shapes_agree(pic, variant):
    cfg = W.scaled(W.config("c1", precision="fp64"), 30_000)
    ref, h = pic.pic_init(cfg), pic.pic_init(cfg)
    assert pic.pic_tune(h, 0, [variant, variant]) == [variant, variant]
    assert pic.pic_step(ref, 3) == 0
    assert pic.pic_step(h, 3) == 0
    same_state(pic, ref, h, 1e-11, exact_ids=True)
    assert list(pic.pic_moments(ref)["counters"][:22]) == list(pic.pic_moments(h)["counters"][:22])


def test_tuner_picks_valid_shapes(pic):
    cfg = W.scaled(W.config("c1"), 50_000)
    h = pic.pic_init(cfg)
    v = pic.pic_tune(h, 1)
    assert all(0 <= x < 4 for x in v)
    assert pic.pic_get_counts(h)["step"] == 4  # one step per shape
    assert pic.pic_step(h, 2) == 0
