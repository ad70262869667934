"""The global X-Y-Z pusher (Sec. 2.3, end) on the CUDA path against the
oracle's (which tests/test_oracle_xyz.py pins to a Cartesian push): one step
with collisions and births, five steps, a_theta included, checkpoint resume.
Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import parity as P
import workloads as W
from oracle import Oracle

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
    s = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a).max() if a.size else 0.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_xyz_one_step_parity(pic, prec):
    cfg = W.config("c1", precision=prec, pusher="xyz")
    for sp in cfg["species"]:
        sp["n_init"] = 0
        sp["capacity"] = 200_000
    rng = np.random.default_rng(4)
    parts = []
    for s, (hot, acc) in enumerate([(3.0, 2e14), (30.0, 5e9)]):
        p = W.random_particles(cfg, s, 30_000, seed=40 + s, hot=hot, accel=acc, wscale=1.5e6)
        k = 3000
        p["r"][:k] = rng.uniform(0.0, 2e-4, k)  # next to the axis
        p["at"] = rng.normal(0.0, acc, 30_000)
        parts.append(p)
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    for s in (0, 1):
        pic.pic_set_particles(h, s, parts[s])
        o.set_particles(s, parts[s])
        o.set_at(s, parts[s]["at"])
    pic.pic_set_step(h, 9)
    o.set_step(9)
    assert pic.pic_step(h, 1) == 0
    o.step(1)
    tol = 1e-12 if prec == "fp64" else 2e-5
    grids = {k: o.grid(k) for k in ("Ez", "Er")}
    o.finalize()
    f = pic.pic_get_fields(h)
    assert nerr(f["phi"], o.grid("phi")) < (tol if prec == "fp64" else 1e-6)
    for s in (0, 1):
        g = pic.pic_get_particles(h, s)
        ref = o.get_particles(s)
        ref["at"] = o.get_at(s)
        # element by element, a_theta in the acceleration vector (tests/parity.py);
        # mixed: each threshold flip explained by FP32 rounding of the inputs
        P.compare_species(cfg, s, g, ref, prec, inputs=parts[s], grids=grids, step=9)


def test_xyz_multi_step_parity_fp64(pic):
    cfg = W.scaled(W.config("c1", precision="fp64", pusher="xyz"), 20_000)
    h = pic.pic_init(cfg)
    o = Oracle(cfg)
    o.load()
    pic.pic_step(h, 5)
    o.step(5)
    f = pic.pic_get_fields(h)
    assert nerr(f["phi"], o.grid("phi")) < 1e-11
    for s in (0, 1):
        g = by_id(pic.pic_get_particles(h, s))
        ref = o.get_particles(s)
        ref["at"] = o.get_at(s)
        ref = by_id(ref)
        assert np.array_equal(g["id"], ref["id"])
        e = P.errors(cfg, s, g, ref, P.e_max({k: o.grid(k) for k in ("Ez", "Er")}), P.w_ref_table(cfg, s))
        assert e.max() < 1e-10, (s, float(e.max()))
        assert np.abs(ref["at"]).max() > 0  # a_theta grew from the rotations


def test_xyz_differs_from_local_and_resumes_from_a_checkpoint(pic, tmp_path):
    base = W.scaled(W.config("c1", precision="fp64"), 20_000)
    xyz = dict(base, pusher="xyz")
    a, b = pic.pic_init(base), pic.pic_init(xyz)
    pic.pic_step(a, 4)
    pic.pic_step(b, 4)
    pa, pb = by_id(pic.pic_get_particles(a, 0)), by_id(pic.pic_get_particles(b, 0))
    assert np.abs(pa["at"]).max() == 0.0 and np.abs(pb["at"]).max() > 0.0
    path = str(tmp_path / "xyz.ck")
    pic.pic_save(b, path)
    c = pic.pic_init(xyz, load=False)
    pic.pic_load(c, path)
    pic.pic_step(b, 3)
    pic.pic_step(c, 3)
    for s in (0, 1):
        u, v = by_id(pic.pic_get_particles(b, s)), by_id(pic.pic_get_particles(c, s))
        assert np.array_equal(u["id"], v["id"])
        for k in FIELDS + ("at",):
            assert nerr(v[k], u[k]) < 1e-12, (s, k)
    with pytest.raises(pic.PicError):
        pic.pic_load(pic.pic_init(base, load=False), path)
