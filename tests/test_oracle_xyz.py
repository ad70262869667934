"""Pin of the oracle's global X-Y-Z pusher (Sec. 2.3, end): one particle pass
in a uniform field against the same D1 pushes written out in Cartesian
coordinates, particle by particle (azimuth 0 at the start; the field's
Cartesian components from E_r along the particle's radius).  Covers the
a_theta the X-Y-Z form carries and the passage through the axis."""
import numpy as np

import workloads as W
from oracle import Oracle


def _cfg():
    cfg = W.collisionless(W.config("c1"))
    cfg["pusher"] = "xyz"
    return cfg


def _cartesian(cfg, s, p, at, Ez0, Er0):
    """Final push at the gathered (uniform) E, walls, first push, walls; the
    result in the particle's new local frame.  None when it left."""
    sp = cfg["species"][s]
    qm, dt = sp["q"] / sp["m"], cfg["dt"]
    L, R = cfg["L"], cfg["R"]
    x = np.array([p["r"], 0.0, p["z"]])
    v = np.array([p["vr"], p["vt"], p["vz"]])
    a = np.array([p["ar"], at, p["az"]])
    E = np.array([Er0, 0.0, Ez0])          # E_r along the radius at azimuth 0
    x1 = x + 0.5 * qm * E * dt * dt
    v1 = v + 0.5 * qm * E * dt
    a1 = 0.5 * (qm * E + a)
    if x1[2] <= 0 or x1[2] >= L or np.hypot(x1[0], x1[1]) >= R:
        return None
    v2 = v1 + 0.5 * a1 * dt
    x2 = x1 + v2 * dt
    r2 = np.hypot(x2[0], x2[1])
    if x2[2] <= 0 or x2[2] >= L or r2 >= R:
        return None
    er = x2[:2] / r2
    et = np.array([-er[1], er[0]])
    return dict(r=r2, z=x2[2], vr=v2[:2] @ er, vt=v2[:2] @ et, vz=v2[2], ar=a1[:2] @ er,
                at=a1[:2] @ et, az=a1[2])


def test_xyz_pusher_is_the_cartesian_push():
    cfg = _cfg()
    n = 400
    rng = np.random.default_rng(5)
    for s, (Ez0, Er0) in enumerate([(2e4, 1e5), (-3e4, -2e5)]):
        p = W.random_particles(cfg, s, n, seed=10 + s, hot=2.0, accel=1e13 if s == 0 else 1e9, margin=1e-3)
        # a quarter of them next to the axis, so that the final push takes
        # them through it
        k = n // 4
        p["r"][:k] = rng.uniform(0.0, 3e-4, k)
        at = rng.normal(0.0, 1e13 if s == 0 else 1e9, n)
        o = Oracle(cfg)
        o.set_particles(s, p)
        o.set_at(s, at)
        o.set_grid("Ez", np.full((cfg["nz"], cfg["nr"]), Ez0))
        o.set_grid("Er", np.full((cfg["nz"], cfg["nr"]), Er0))
        o.particle_pass()
        got = o.get_particles(s)
        gat = o.get_at(s)
        by = {int(i): q for q, i in enumerate(got["id"])}
        crossed = 0
        for q in range(n):
            ref = _cartesian(cfg, s, {f: p[f][q] for f in ("r", "z", "vr", "vt", "vz", "ar", "az")},
                             at[q], Ez0, Er0)
            sp = cfg["species"][s]
            rr = p["r"][q] + 0.5 * sp["q"] / sp["m"] * Er0 * cfg["dt"] ** 2
            crossed += rr < 0
            if ref is None:
                assert int(p["id"][q]) not in by
                continue
            g = by[int(p["id"][q])]
            for f in ("r", "z", "vr", "vt", "vz", "ar", "az"):
                assert abs(got[f][g] - ref[f]) <= 1e-12 * max(abs(ref[f]), 1e-300) + 1e-15, (s, q, f)
            assert abs(gat[g] - ref["at"]) <= 1e-12 * abs(ref["at"]) + 1e-3, (s, q)
        if s == 0:
            assert crossed > 50  # the axis passage was exercised


def test_local_pusher_drops_a_theta():
    cfg = W.collisionless(W.config("c1"))
    p = W.random_particles(cfg, 1, 200, seed=3, hot=2.0, accel=1e9, margin=1e-3)
    o = Oracle(cfg)
    o.set_particles(1, p)
    o.set_at(1, np.full(200, 1e9))
    o.set_grid("Ez", np.full((cfg["nz"], cfg["nr"]), 1e4))
    o.set_grid("Er", np.full((cfg["nz"], cfg["nr"]), 1e4))
    o.particle_pass()
    # the local form keeps the set a_theta out of the push: halved by the
    # final push, never rotated in
    ref = Oracle(cfg)
    ref.set_particles(1, p)
    ref.set_grid("Ez", np.full((cfg["nz"], cfg["nr"]), 1e4))
    ref.set_grid("Er", np.full((cfg["nz"], cfg["nr"]), 1e4))
    ref.particle_pass()
    a, b = o.get_particles(1), ref.get_particles(1)
    for f in ("r", "z", "vr", "vt", "vz", "ar", "az"):
        assert np.array_equal(a[f], b[f])
