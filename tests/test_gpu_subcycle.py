"""Ion subcycling (Sec. 2.7) on the CUDA path, through the C ABI, against
the oracle's (tests/test_oracle_subcycle.py pins it): a pass that holds the
ions and one that moves them, with collisions and births; ten steps through
both kinds with a split; the same run cut into several calls and launched
without graphs; a checkpoint taken while newborn ions wait for their next
moving pass; the particle-step count; the refusals.
Tolerances as in test_gpu_parity.py, element by element (tests/parity.py):
FP64 1e-12 per step, 1e-10 over ten steps; mixed 2e-5, every threshold flip
explained by FP32 rounding of the inputs."""
import numpy as np
import pytest

import parity as P
import workloads as W
from oracle import C_ABS, C_BIRTHS, C_CAND, C_COLL, C_SPLITS, Oracle

pytestmark = pytest.mark.gpu

K = 4
FIELDS = ("r", "z", "vr", "vt", "vz", "ar", "az", "w")
TOL = {"fp64": 1e-12, "mixed": 2e-5}


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


def _cfg(prec, split_every=0, capacity=400_000):
    cfg = W.config("c1", precision=prec, ion_subcycle=K, split_every=split_every)
    for sp in cfg["species"]:
        sp["n_init"] = 0
        sp["capacity"] = capacity
    return cfg


def _state(cfg, n_e, n_i, seed):
    e = W.random_particles(cfg, 0, n_e, seed=seed, hot=3.0, accel=2e14, wscale=1.5e6)
    i = W.random_particles(cfg, 1, n_i, seed=seed + 1, hot=30.0, accel=5e9, wscale=1.5e6)
    return e, i


def _pair(pic, cfg, e, i, step0):
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    for s, p in ((0, e), (1, i)):
        pic.pic_set_particles(h, s, p)
        o.set_particles(s, p)
    pic.pic_set_step(h, step0)
    o.set_step(step0)
    return h, o


def _compare(pic, cfg, h, o, prec, tol_p, tol_f, inputs=None, step0=None):
    f = pic.pic_get_fields(h)
    grids = {k: o.grid(k) for k in ("Ez", "Er")}
    o.finalize()
    for name in ("phi", "Ez", "Er"):
        assert nerr(f[name], o.grid(name)) < tol_f, name
    for name in ("rho", "chi"):
        assert nerr(f[name], o.grid(name)) < (tol_f if prec == "fp64" else 5e-5), name
    for s in (0, 1):
        g, ref = pic.pic_get_particles(h, s), o.get_particles(s)
        if prec == "fp64":
            gs, rs = by_id(g), by_id(ref)
            assert np.array_equal(gs["id"], rs["id"]), s
            P.check_sorted(g, (cfg["nz"] - 1) * (cfg["nr"] - 1))
            e = P.errors(cfg, s, gs, rs, P.e_max(grids), P.w_ref_table(cfg, s))
            assert e.max(initial=0.0) <= tol_p, (s, float(e.max(initial=0.0)))
        else:
            P.compare_species(cfg, s, g, ref, prec, inputs=inputs[s], grids=grids, step=step0)
    m = pic.pic_moments(h)
    oc, oq = o.counters()
    idx = list(range(C_COLL, C_COLL + 8)) + [C_CAND, C_CAND + 1, C_BIRTHS, C_BIRTHS + 1,
                                              C_SPLITS, C_SPLITS + 1] + list(range(C_ABS, C_ABS + 6))
    for k in idx:
        if prec == "fp64":
            assert m["counters"][k] == oc[k], (k, m["counters"][k], oc[k])
        else:
            assert abs(int(m["counters"][k]) - int(oc[k])) <= max(3, 1e-4 * oc[k]), k
    if prec == "fp64":
        assert list(pic.pic_get_counts(h)["next_id"]) == [o.next_id(0), o.next_id(1)]
        for k in ("ne", "ni"):
            assert nerr(m[k], o.moments()[k]) < 1e-10, k
    return oc


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("step0", [K - 1, 1])
def test_one_pass_that_moves_or_holds_the_ions(pic, prec, step0):
    cfg = _cfg(prec)
    e, i = _state(cfg, 60_001, 40_003, seed=5)
    h, o = _pair(pic, cfg, e, i, step0)
    assert pic.pic_step(h, 1) == 0
    o.step(1)
    oc = _compare(pic, cfg, h, o, prec, TOL[prec], TOL[prec] if prec == "fp64" else 1e-6, inputs=(e, i),
                  step0=step0)
    assert oc[C_COLL + 2] > 50  # ionisations: newborn ions in both kinds of pass
    if step0 == K - 1:
        assert oc[C_COLL + 4] > 0  # the moving pass has charge exchange
    else:
        assert oc[C_CAND + 1] == 0  # held ions are not candidates


def test_ten_steps_through_both_kinds_with_a_split_fp64(pic):
    cfg = _cfg("fp64", split_every=2 * K)
    e, i = _state(cfg, 30_000, 20_000, seed=11)
    i["w"] = i["w"] * 20.0  # heavy ions near the axis split
    h, o = _pair(pic, cfg, e, i, 1)
    assert pic.pic_step(h, 10) == 0  # passes 1..10: moving ones 3 and 7, split at 7
    o.step(10)
    oc = _compare(pic, cfg, h, o, "fp64", 1e-10, 1e-11)
    assert oc[C_SPLITS + 1] > 0 and oc[C_COLL + 4] > 0


def test_calls_and_launch_modes_give_the_same_run(pic):
    """One call of nine steps, the same steps cut into calls of 2, 3, 1 and
    3 (the held ions are sorted at each call's end and again before their
    next moving pass), and the steps launched one by one: the same ids and
    counts, states to rounding (deposit atomics add in any order)."""
    cfg = _cfg("fp64")
    e, i = _state(cfg, 20_000, 20_000, seed=17)
    runs = []
    for mode in ("one", "cut", "direct"):
        h, _ = _pair(pic, cfg, e, i, 0)
        if mode == "direct":
            pic.pic_profile(h, True)
        for n in ((9,) if mode != "cut" else (2, 3, 1, 3)):
            assert pic.pic_step(h, n) == 0
        runs.append(h)
    ref = [by_id(pic.pic_get_particles(runs[0], s)) for s in (0, 1)]
    c0 = pic.pic_moments(runs[0])["counters"]
    for h in runs[1:]:
        # every counter but the multigrid cycles (rounding may move one) and the steps
        assert np.array_equal(pic.pic_moments(h)["counters"][:22], c0[:22])
        for s in (0, 1):
            g = by_id(pic.pic_get_particles(h, s))
            assert np.array_equal(g["id"], ref[s]["id"])
            for k in FIELDS:
                assert nerr(g[k], ref[s][k]) < 1e-12, (s, k)


def test_checkpoint_while_newborn_ions_wait(pic, tmp_path):
    cfg = _cfg("fp64")
    e, i = _state(cfg, 20_000, 20_000, seed=23)
    a, _ = _pair(pic, cfg, e, i, 0)
    assert pic.pic_step(a, 5) == 0  # moving pass 3; passes 4 and 5 hold: newborns wait
    path = str(tmp_path / "sub.ck")
    pic.pic_save(a, path)
    b = pic.pic_init(cfg, load=False)
    pic.pic_load(b, path)
    assert pic.pic_step(a, 4) == 0
    assert pic.pic_step(b, 4) == 0
    for s in (0, 1):
        u, v = by_id(pic.pic_get_particles(a, s)), by_id(pic.pic_get_particles(b, s))
        assert np.array_equal(u["id"], v["id"])
        for k in FIELDS:
            assert nerr(v[k], u[k]) < 1e-12, (s, k)
    other = dict(cfg, ion_subcycle=2)
    with pytest.raises(pic.PicError):
        pic.pic_load(pic.pic_init(other, load=False), path)


def test_births_overflow_in_a_holding_pass_keeps_the_last_completed_step(pic):
    """Held ions collect newborns over passes 0, 1 and 2 (about 400 a pass
    here) in a births buffer of 900: pass 2 overflows it, the call fails
    with the capacity status, and the state is the one after pass 1 -- the
    ions' births, counts, order and deposit included."""
    cfg = dict(_cfg("fp64"), births_capacity=900)
    e, i = _state(cfg, 60_001, 40_003, seed=5)
    h, _ = _pair(pic, cfg, e, i, 0)
    ref, _ = _pair(pic, _cfg("fp64"), e, i, 0)
    with pytest.raises(pic.PicError) as err:
        pic.pic_step(h, 3)
    assert err.value.status == pic.PIC_ERR_CAPACITY
    assert pic.pic_step(ref, 2) == 0
    assert pic.pic_get_counts(h)["step"] == 2
    assert list(pic.pic_get_counts(h)["n_alive"]) == list(pic.pic_get_counts(ref)["n_alive"])
    for s in (0, 1):
        u, v = by_id(pic.pic_get_particles(ref, s)), by_id(pic.pic_get_particles(h, s))
        assert np.array_equal(u["id"], v["id"]), s
        for k in FIELDS:
            assert nerr(v[k], u[k]) < 1e-12, (s, k)
    fh, fr = pic.pic_get_fields(h), pic.pic_get_fields(ref)
    for name in ("rho", "chi"):
        assert nerr(fh[name], fr[name]) < 1e-12, name


def test_particle_steps_count_moved_ions_only(pic):
    cfg = W.collisionless(_cfg("fp64"))
    n = 10_000
    e = W.random_particles(cfg, 0, n, seed=3, hot=0.05, margin=3e-3, wscale=1e5)
    i = W.random_particles(cfg, 1, n, seed=4, hot=1.0, margin=3e-3, wscale=1e5)
    h, _ = _pair(pic, cfg, e, i, 0)
    assert pic.pic_step(h, 2 * K + 1) == 0
    assert list(pic.pic_get_counts(h)["n_alive"]) == [n, n]
    assert int(pic.pic_moments(h)["counters"][pic.PIC_C_PSTEPS]) == (2 * K + 1) * n + 2 * n


def test_refusals(pic):
    with pytest.raises(pic.PicError):
        pic.pic_init(dict(_cfg("fp64"), ion_subcycle=3, split_every=400), load=False)
    h = pic.pic_init(_cfg("fp64"), load=False)
    with pytest.raises(pic.PicError):
        pic.pic_batch_init([h])
    w = np.ones((33, 65))
    with pytest.raises(pic.PicError):
        pic.pic_window(h, 2, 1, w, 100.0)
