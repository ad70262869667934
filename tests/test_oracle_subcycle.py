"""Pins of the oracle's ion subcycling (Sec. 2.7, Vahedi's method; the form
for the implicit scheme is a reading: ions move in the passes n with
n mod K = K - 1, with dt_i = K dt, and are held still otherwise).

- a moving pass is one D1 pass with dt_i: the same pushes written out in
  Cartesian coordinates in a uniform field, particle by particle;
- a holding pass leaves the ions' state and deposit exactly as they were;
- the ions' susceptibility carries dt_i^2 before a moving pass and is
  absent before a holding one (chi is quadratic in the step);
- the ions' null-collision candidates follow P_null = 1 - exp(-nu_max dt_i)
  (binomial bound);
- ions born from electrons take their first push with dt_i: walking each
  newborn ion back along its straight line for dt_i lands on its parent's
  position (a zero field, no accelerations);
- K = 1 is the plain method, bit for bit.
"""
import numpy as np

import workloads as W
from oracle import C_BIRTHS, C_CAND, Oracle


def _ions_only(cfg, n, seed, hot=3.0, accel=1e9, margin=2e-3):
    p = W.random_particles(cfg, 1, n, seed=seed, hot=hot, accel=accel, margin=margin)
    return p


def _cartesian(cfg, s, p, Ez0, Er0, dt):
    """Final push in a uniform field, walls, first push, walls (Cartesian,
    azimuth 0 at the start; a_theta = 0 and dropped as the local pusher
    does).  None when the particle left."""
    sp = cfg["species"][s]
    qm = sp["q"] / sp["m"]
    L, R = cfg["L"], cfg["R"]
    x = np.array([p["r"], 0.0, p["z"]])
    v = np.array([p["vr"], p["vt"], p["vz"]])
    a = np.array([p["ar"], 0.0, p["az"]])
    E = np.array([Er0, 0.0, Ez0])
    x1 = x + 0.5 * qm * E * dt * dt
    v1 = v + 0.5 * qm * E * dt
    a1 = 0.5 * (qm * E + a)
    if x1[2] <= 0 or x1[2] >= L or x1[0] >= R:
        return None
    v2 = v1 + 0.5 * a1 * dt
    x2 = x1 + v2 * dt
    r2 = np.hypot(x2[0], x2[1])
    if x2[2] <= 0 or x2[2] >= L or r2 >= R:
        return None
    er = x2[:2] / r2
    et = np.array([-er[1], er[0]])
    return dict(r=r2, z=x2[2], vr=v2[:2] @ er, vt=v2[:2] @ et, vz=v2[2], ar=a1[:2] @ er, az=a1[2])


def _uniform(o, cfg, Ez0, Er0):
    o.set_grid("Ez", np.full((cfg["nz"], cfg["nr"]), Ez0))
    o.set_grid("Er", np.full((cfg["nz"], cfg["nr"]), Er0))


def test_moving_pass_is_one_d1_pass_with_dt_i_and_holding_pass_keeps_the_ions():
    K = 4
    cfg = dict(W.collisionless(W.config("c1")), ion_subcycle=K)
    n = 300
    p = _ions_only(cfg, n, seed=3)
    # kept away from the axis: the final push never reaches it here
    p["r"] = np.maximum(p["r"], 3e-3)
    Ez0, Er0 = 3e4, -2e4
    o = Oracle(cfg)
    o.set_particles(1, p)
    _uniform(o, cfg, Ez0, Er0)
    o.deposit()
    N0 = o.grid("Ni")
    # passes 0 .. K-2 hold the ions: state and deposit unchanged, bit for bit
    for step in range(K - 1):
        o.set_step(step)
        assert not o.ion_pass()
        o.particle_pass()
        o.deposit()
        got = o.get_particles(1)
        o_ = np.argsort(got["id"])
        ref = np.argsort(p["id"])
        for f in ("r", "z", "vr", "vt", "vz", "ar", "az", "w"):
            assert np.array_equal(got[f][o_], p[f][ref]), f
        assert np.array_equal(o.grid("Ni"), N0)
    # pass K-1 moves them with dt_i = K dt
    o.set_step(K - 1)
    assert o.ion_pass()
    o.particle_pass()
    got = o.get_particles(1)
    by = {int(i): q for q, i in enumerate(got["id"])}
    dti = K * cfg["dt"]
    moved = 0
    for q in range(n):
        ref = _cartesian(cfg, 1, {f: p[f][q] for f in ("r", "z", "vr", "vt", "vz", "ar", "az")}, Ez0, Er0, dti)
        if ref is None:
            assert int(p["id"][q]) not in by
            continue
        g = by[int(p["id"][q])]
        for f in ref:
            assert abs(got[f][g] - ref[f]) <= 1e-12 * max(abs(ref[f]), 1e-300) + 1e-15, (q, f)
        moved += 1
    assert moved > n // 2


def test_chi_carries_dt_i_squared_before_a_moving_pass_only():
    base = W.collisionless(W.config("c1"))
    p = _ions_only(base, 5000, seed=5)
    chis, rhos = {}, {}
    for K, step in ((1, 0), (3, 2), (3, 0), (3, 1)):
        o = Oracle(dict(base, ion_subcycle=K))
        o.set_particles(1, p)
        o.deposit()
        o.set_step(step)
        o.finalize()
        chis[K, step] = o.grid("chi")
        rhos[K, step] = o.grid("rho")
    ref = chis[1, 0]
    assert ref.max() > 0
    assert np.allclose(chis[3, 2], 9.0 * ref, rtol=1e-14, atol=0)
    assert np.array_equal(chis[3, 0], np.zeros_like(ref))
    assert np.array_equal(chis[3, 1], np.zeros_like(ref))
    for key in rhos:
        assert np.array_equal(rhos[key], rhos[1, 0])


def test_ion_candidates_follow_p_null_of_dt_i():
    cfg0 = W.config("c1")
    n = 200_000
    p = _ions_only(cfg0, n, seed=9, hot=1.0, accel=0.0, margin=1e-3)
    seen = {}
    for K in (1, 4):
        cfg = dict(cfg0, ion_subcycle=K, split_every=0)
        o = Oracle(cfg, capacity=2 * n)
        o.set_particles(1, p)
        _uniform(o, cfg, 0.0, 0.0)
        o.set_step(K - 1)
        o.particle_pass()
        c, _ = o.counters()
        nu_dt = o.nu_max(1) * K * cfg["dt"]
        P = 1.0 - np.exp(-nu_dt)
        sd = np.sqrt(n * P * (1 - P))
        assert abs(c[C_CAND + 1] - n * P) < 4 * sd, (K, c[C_CAND + 1], n * P, sd)
        seen[K] = c[C_CAND + 1]
    assert seen[4] > 3 * seen[1]


def test_newborn_ions_take_their_first_push_with_dt_i():
    """Electrons that ionise in a zero field, accelerations zero: a newborn
    ion starts at its parent's position with the gas atom's velocity and
    moves on a straight line for dt_i.  Walking it back by dt_i in its own
    frame lands on a parent electron's position (to rounding); walking it
    back by dt does not."""
    K = 5
    cfg = W.config("c1")
    xs = [dict(t) for t in cfg["xsec"]]
    sig = np.array(xs[0]["sigma"], dtype=np.float64).copy()
    sig[0] = 0.0  # no elastic
    sig[1] = 0.0  # no excitation: the electrons' real collisions ionise
    xs[0]["sigma"] = sig
    xs[1] = dict(xs[1], sigma=np.zeros_like(np.asarray(xs[1]["sigma"], dtype=np.float64)))
    cfg = dict(cfg, xsec=xs, ion_subcycle=K, split_every=0)
    n = 20_000
    e = W.random_particles(cfg, 0, n, seed=21, hot=3.5, accel=0.0, margin=2e-3)
    for step in (0, K - 1):  # a holding pass and a moving one: newborns alike
        o = Oracle(cfg, capacity=4 * n)
        o.set_particles(0, e)
        o.set_next_id(1, 10**9)
        _uniform(o, cfg, 0.0, 0.0)
        o.set_step(step)
        o.particle_pass()
        c, _ = o.counters()
        ions = o.get_particles(1)
        nb = len(ions["id"])
        assert nb == c[C_BIRTHS + 1] - 0 and nb > 50, nb
        parents = np.stack([e["r"], e["z"]], axis=1)
        for dt_back, must_hit in ((K * cfg["dt"], True), (cfg["dt"], False)):
            r0 = np.hypot(ions["r"] - ions["vr"] * dt_back, ions["vt"] * dt_back)
            z0 = ions["z"] - ions["vz"] * dt_back
            d = np.min(np.abs(parents[None, :, 0] - r0[:, None]) + np.abs(parents[None, :, 1] - z0[:, None]), axis=1)
            if must_hit:
                assert d.max() < 1e-12, d.max()
            else:
                assert np.median(d) > 1e-9, np.median(d)


def test_k1_is_the_plain_method():
    cfg = W.scaled(W.config("c1"), 20_000)
    a, b = Oracle(cfg), Oracle(dict(cfg, ion_subcycle=1))
    a.load()
    b.load()
    a.step(3)
    b.step(3)
    for s in (0, 1):
        pa, pb = a.get_particles(s), b.get_particles(s)
        for f in pa:
            assert np.array_equal(pa[f], pb[f]), (s, f)
    assert np.array_equal(a.grid("phi"), b.grid("phi"))
