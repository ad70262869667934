"""Pins of the oracle's pusher (closed forms) and weighting (invariants, lattice loads)."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle


def _vacuum(cfg):
    """No gas (no collisions) and no splitting."""
    cfg = dict(cfg)
    cfg["gas"] = dict(cfg["gas"], p_Pa=0.0)
    cfg["split_every"] = 0
    return cfg


def _state(n, **kw):
    base = dict(r=np.zeros(n), z=np.zeros(n), vr=np.zeros(n), vt=np.zeros(n), vz=np.zeros(n),
                ar=np.zeros(n), az=np.zeros(n), w=np.ones(n), id=np.arange(n, dtype=np.uint64))
    for k, v in kw.items():
        base[k] = np.broadcast_to(np.asarray(v, dtype=base[k].dtype), (n,)).copy()
    return base


def _fields(o, Ez=0.0, Er=0.0):
    shape = (o.nz, o.nr)
    o.set_grid("Ez", np.full(shape, Ez))
    o.set_grid("Er", np.full(shape, Er))


def test_uniform_field_is_leapfrog_closed_form():
    """D1 with a constant acceleration a and a_bar = a reduces to leapfrog (Sec. 2.1):
    x^n = x^0 + n v^{-1/2} dt + a dt^2 n(n+1)/2."""
    cfg = _vacuum(W.config("c1"))
    o = Oracle(cfg)
    s, sp = 0, cfg["species"][0]
    dt = cfg["dt"]
    Ez = 2000.0
    a = sp["q"] / sp["m"] * Ez
    n = 8
    z0 = np.linspace(0.006, 0.014, n)
    r0 = np.linspace(0.005, 0.04, n)
    vm = np.linspace(-3e4, 3e4, n)  # v^{-1/2}
    # stored state after the first push: x~^1 = x^0 + (v^{-1/2} + a dt/2) dt, a_bar = a
    vt = vm + 0.5 * a * dt
    st = _state(n, r=r0, z=z0 + vt * dt, vz=vt, az=a)
    o.set_particles(s, st)
    o.set_particles(1, _state(0))
    _fields(o, Ez=Ez)
    K = 12
    for _ in range(K):
        o.particle_pass()
    p = o.get_particles(s)
    order = np.argsort(p["id"])
    # stored x~^{K+1} = x^K + v~^{K+1/2} dt, v~^{K+1/2} = v^{-1/2} + K a dt + a dt/2
    xK = z0 + K * vm * dt + a * dt * dt * K * (K + 1) / 2
    vK = vm + K * a * dt + 0.5 * a * dt
    np.testing.assert_allclose(p["z"][order], xK + vK * dt, rtol=1e-13, atol=1e-17)
    np.testing.assert_allclose(p["vz"][order], vK, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(p["az"][order], a, rtol=1e-14)
    np.testing.assert_allclose(p["r"][order], r0, rtol=1e-15)


def test_local_xy_frame_straight_line_is_exact():
    """Field-free motion in the local X-Y frame with theta rotation (Sec. 2.3) is an exact
    straight line: r(t) = sqrt((r0 + v_r t)^2 + (v_theta t)^2), r v_theta conserved."""
    cfg = _vacuum(W.config("c1"))
    o = Oracle(cfg)
    dt = cfg["dt"]
    n = 6
    r0 = np.array([1e-3, 5e-3, 2e-2, 3e-4, 1e-3, 4e-3])
    vr = np.array([2e5, -3e5, 1e5, -4e5, -2e6, 0.0])
    vt = np.array([1e5, 2e5, -3e5, 5e4, 0.0, 3e5])
    st = _state(n, r=r0, z=0.01, vr=vr, vt=vt)
    o.set_particles(0, st)
    o.set_particles(1, _state(0))
    _fields(o)
    K = 7
    for _ in range(K):
        o.particle_pass()
    p = o.get_particles(0)
    order = np.argsort(p["id"])
    t = K * dt
    x, y = r0 + vr * t, vt * t
    rK = np.hypot(x, y)
    np.testing.assert_allclose(p["r"][order], rK, rtol=1e-12)
    np.testing.assert_allclose((p["r"] * p["vt"])[order], r0 * vt, rtol=1e-11, atol=1e-9)
    speed = np.hypot(p["vr"], p["vt"])[order]
    np.testing.assert_allclose(speed, np.hypot(vr, vt), rtol=1e-12)
    # straight through the axis (v_theta = 0): |r0 + v_r t| and v_r flips sign
    assert p["vr"][order][4] > 0


def test_axis_crossing_in_final_push_takes_absolute_values():
    """A particle pushed through r = 0 by the final push gets |r|, |v_r|, |a_r| (Sec. 2.3)."""
    cfg = _vacuum(W.config("c1"))
    o = Oracle(cfg)
    sp = cfg["species"][0]
    dt = cfg["dt"]
    Er = 4e4  # electrons accelerate towards -r
    a = sp["q"] / sp["m"] * Er
    r0 = 1e-5
    o.set_particles(0, _state(1, r=r0, z=0.01))
    o.set_particles(1, _state(0))
    _fields(o, Er=Er)
    o.particle_pass()
    p = o.get_particles(0)
    r2 = abs(r0 + 0.5 * a * dt * dt)
    v2 = abs(0.5 * a * dt)
    a2 = abs(0.5 * a)
    assert r0 + 0.5 * a * dt * dt < 0
    # then the first push: v_x = v + a dt/2, x = r + v_x dt (v_theta = 0: no rotation)
    vx = v2 + 0.5 * a2 * dt
    np.testing.assert_allclose(p["r"][0], r2 + vx * dt, rtol=1e-13)
    np.testing.assert_allclose(p["vr"][0], vx, rtol=1e-13)
    np.testing.assert_allclose(p["ar"][0], a2, rtol=1e-13)


def test_walls_absorb_and_count_charge():
    cfg = _vacuum(W.config("c1"))
    o = Oracle(cfg)
    L, R, dt = cfg["L"], cfg["R"], cfg["dt"]
    q = cfg["species"][0]["q"]
    st = _state(3, r=[0.01, 0.01, R - 1e-6], z=[1e-7, L - 1e-7, 0.01],
                vz=[-1e4, 1e4, 0.0], vr=[0.0, 0.0, 1e4], w=[1.0, 2.0, 4.0])
    o.set_particles(0, st)
    o.set_particles(1, _state(0))
    _fields(o)
    o.particle_pass()
    assert o.count(0) == 0
    c, qa = o.counters()
    np.testing.assert_allclose(qa, [q * 1.0, q * 2.0, q * 4.0], rtol=1e-15)


@pytest.mark.parametrize("weighting", ["zr2", "zr"])
def test_deposit_conserves_total_weight(weighting):
    cfg = W.config("c1", weighting=weighting)
    o = Oracle(cfg)
    for s in (0, 1):
        o.set_particles(s, W.random_particles(cfg, s, 20000, seed=11 + s))
    o.deposit()
    for s, name in ((0, "Ne"), (1, "Ni")):
        w = o.get_particles(s)["w"]
        assert abs(o.grid(name).sum() / w.sum() - 1) < 1e-13


def _lattice(cfg, weighting, n0, m=3):
    """Deterministic load of uniform density n0 whose node sums are exact for the shape
    functions: midpoints in (z, r^2) for z-r^2; 2-point Gauss-Legendre in r with weights
    proportional to r for z-r (exact for the quadratic r S_r(r))."""
    nz, nr, L, R = cfg["nz"], cfg["nr"], cfg["L"], cfg["R"]
    dz, dr = L / (nz - 1), R / (nr - 1)
    zs, rs, ws = [], [], []
    for i in range(nz - 1):
        for a in range(m):
            za, zb = i * dz + a * dz / m, i * dz + (a + 1) * dz / m
            zc = 0.5 * (za + zb)
            for j in range(nr - 1):
                for b in range(m):
                    ra, rb = j * dr + b * dr / m, j * dr + (b + 1) * dr / m
                    if weighting == "zr2":
                        rp = np.sqrt(0.5 * (ra * ra + rb * rb))
                        zs.append(zc)
                        rs.append(rp)
                        ws.append(n0 * np.pi * (rb * rb - ra * ra) * (zb - za))
                    else:
                        c, h = 0.5 * (ra + rb), 0.5 * (rb - ra)
                        for sgn in (-1, 1):
                            rp = c + sgn * h / np.sqrt(3.0)
                            zs.append(zc)
                            rs.append(rp)
                            ws.append(n0 * 2 * np.pi * rp * h * (zb - za))
    n = len(zs)
    return dict(r=np.array(rs), z=np.array(zs), vr=np.zeros(n), vt=np.zeros(n), vz=np.zeros(n),
                ar=np.zeros(n), az=np.zeros(n), w=np.array(ws), id=np.arange(n, dtype=np.uint64))


@pytest.mark.parametrize("weighting", ["zr2", "zr"])
def test_uniform_density_recovered_including_axis(weighting):
    """Node volumes of Sec. 2.4 turn a uniform load into n0 at every interior node,
    the axis node j = 0 included (its own V_0 per weighting)."""
    cfg = W.config("c1", weighting=weighting, nz=9, nr=17)
    n0 = 3e15
    o = Oracle(cfg)
    o.set_particles(0, _lattice(cfg, weighting, n0))
    o.set_particles(1, _state(0))
    o.deposit()
    n = o.grid("Ne") / o.node_volumes()
    inner = n[1:-1, :-1]
    np.testing.assert_allclose(inner, n0, rtol=1e-12)
    # boundary rows and the r = R column hold the inside half of the support
    np.testing.assert_allclose(n[0, :-1], n0, rtol=1e-12)
    np.testing.assert_allclose(n[1:-1, -1], n0, rtol=1e-12)
