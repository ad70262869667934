"""Pins of the oracle's null-collision Monte Carlo (Sec. 2.6), weight splitting (Sec. 2.2)
and whole-step invariants."""
import numpy as np
import pytest

import workloads as W
from oracle import C_ABS, C_BIRTHS, C_CAND, C_COLL, C_SPLITS, Oracle, ejected_energy, scatter_dir

QE, ME, MAR, KB = W.QE, W.ME, W.M_AR, W.KB


def _state(n, **kw):
    base = dict(r=np.full(n, 0.02), z=np.full(n, 0.01), vr=np.zeros(n), vt=np.zeros(n),
                vz=np.zeros(n), ar=np.zeros(n), az=np.zeros(n), w=np.ones(n),
                id=np.arange(n, dtype=np.uint64))
    for k, v in kw.items():
        base[k] = np.broadcast_to(np.asarray(v, dtype=base[k].dtype), (n,)).copy()
    return base


def _zero_fields(o):
    o.set_grid("Ez", np.zeros((o.nz, o.nr)))
    o.set_grid("Er", np.zeros((o.nz, o.nr)))


def _sigma_analytic(E):
    """The synthetic argon forms, written out (independent of the tables)."""
    el = 1e-19
    ex = 0.0 if E <= 11.5 else (2e-20 * (E - 11.5) / 13.5 if E <= 25 else 2e-20 * 25 / E)
    iz = 0.0 if E <= 15.76 else (3e-20 * (E - 15.76) / (100 - 15.76) if E <= 100 else 3e-20 * 100 / E)
    return np.array([el, ex, iz])


def test_nu_max_closed_form():
    cfg = W.config("c1")
    o = Oracle(cfg)
    ng = cfg["gas"]["p_Pa"] / (KB * cfg["gas"]["T_K"])
    Emax = cfg["xsec"][0]["E_max"]
    # sigma_tot * sqrt(E) rises up to the end of the table for these forms
    nu_e = ng * _sigma_analytic(Emax).sum() * np.sqrt(2 * Emax * QE / ME)
    assert abs(o.nu_max(0) / (nu_e * (1 + 1e-6)) - 1) < 1e-12
    nu_i = ng * 5e-19 * np.sqrt(2 * Emax * QE / MAR)
    assert abs(o.nu_max(1) / (nu_i * (1 + 1e-6)) - 1) < 1e-12
    assert abs(o.p_null(0) - (1 - np.exp(-o.nu_max(0) * cfg["dt"]))) < 1e-15


def test_candidate_fraction_and_channel_rates():
    """Monoenergetic 60 eV electrons: candidates ~ Binomial(N, P_null); real collisions per
    channel ~ N P_null nu_k(E)/nu_max (null-collision method, Sec. 2.6)."""
    cfg = W.config("c1", split_every=0)
    o = Oracle(cfg, capacity=600_000)
    N = 200_000
    E = 60.0
    v = np.sqrt(2 * E * QE / ME)
    rng = np.random.default_rng(4)
    d = rng.normal(size=(3, N))
    d /= np.linalg.norm(d, axis=0)
    o.set_particles(0, _state(N, vr=v * d[0], vt=v * d[1], vz=v * d[2], r=0.02, z=0.01))
    o.set_particles(1, _state(0))
    _zero_fields(o)
    o.particle_pass()
    c, _ = o.counters()
    P = o.p_null(0)
    sd = np.sqrt(N * P * (1 - P))
    assert abs(c[C_CAND] - N * P) < 4 * sd
    ng = cfg["gas"]["p_Pa"] / (KB * cfg["gas"]["T_K"])
    nu = ng * _sigma_analytic(E) * v
    for ch in range(3):
        p = P * nu[ch] / o.nu_max(0)
        exp = N * p
        assert abs(c[C_COLL + ch] - exp) < 4 * np.sqrt(exp * (1 - p)) + 1, (ch, c[C_COLL + ch], exp)
    # every ionisation made one electron and one ion
    assert c[C_BIRTHS + 0] == c[C_COLL + 2] and c[C_BIRTHS + 1] == c[C_COLL + 2]


def test_vahedi_surendra_angle_mean():
    """E[cos chi] over R of the Vahedi-Surendra law: (2 + e - 2 e / ln(1 + e)) / e."""
    o = Oracle(W.config("c1"))
    M = 20000
    R = (np.arange(M) + 0.5) / M
    for eps in (0.5, 5.0, 50.0, 300.0):
        mean = np.mean([o.cos_chi(eps, x) for x in R])
        exact = (2 + eps - 2 * eps / np.log1p(eps)) / eps
        assert abs(mean - exact) < 1e-6, (eps, mean, exact)


def test_scatter_direction_geometry():
    rng = np.random.default_rng(1)
    for _ in range(200):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        cc = rng.uniform(-1, 1)
        # unit norm and the prescribed polar angle, for any azimuth
        phis = np.linspace(0, 2 * np.pi, 64, endpoint=False)
        outs = np.array([scatter_dir(*u, cc, ph) for ph in phis])
        np.testing.assert_allclose(np.linalg.norm(outs, axis=1), 1.0, rtol=1e-13)
        np.testing.assert_allclose(outs @ u, cc, atol=1e-13)
        # the azimuth sweeps a cone around u: its mean is cos(chi) u
        np.testing.assert_allclose(outs.mean(axis=0), cc * u, atol=1e-13)
    # along the z axis
    out = scatter_dir(0.0, 0.0, -1.0, 0.3, 1.0)
    assert abs(np.linalg.norm(out) - 1) < 1e-14 and abs(out[2] + 0.3) < 1e-14


def test_ionisation_energy_sharing_distribution():
    """Opal's form: ejected energy density ~ 1/(B^2 + x^2) on [0, (E - thr)/2]."""
    E, thr, B = 80.0, 15.76, 10.0
    M = 200_000
    R = (np.arange(M) + 0.5) / M
    x = np.array([ejected_energy(E, thr, B, r) for r in R])
    assert x.min() >= 0 and x.max() <= (E - thr) / 2 + 1e-12
    edges = np.linspace(0, (E - thr) / 2, 17)
    h = np.histogram(x, bins=edges)[0] / M
    cdf = np.arctan(edges / B) / np.arctan((E - thr) / (2 * B))
    np.testing.assert_allclose(h, np.diff(cdf), atol=2e-5)


def test_ionisation_conserves_energy_minus_threshold_and_scales_acceleration():
    cfg = W.config("c1", split_every=0)
    o = Oracle(cfg, capacity=400_000)
    N = 100_000
    E = 90.0
    v = np.sqrt(2 * E * QE / ME)
    a0 = np.array([3e14, -2e14])
    o.set_particles(0, _state(N, vz=v, ar=a0[0], az=a0[1]))
    o.set_particles(1, _state(0))
    _zero_fields(o)
    # one pass: a_bar'' = a/2 (E = 0), then the first push keeps a_z, rotates a_r
    o.particle_pass()
    e = o.get_particles(0)
    ions = o.get_particles(1)
    n_iz = len(ions["r"])
    assert n_iz > 10
    start = o.next_id(0) - n_iz
    new_e = e["id"] >= start
    assert new_e.sum() == n_iz
    # the ion ids are 0..n-1 and follow the parents' id order, like the new electrons'
    assert np.array_equal(np.sort(ions["id"]), np.arange(n_iz, dtype=np.uint64))
    # new ion acceleration: a_e (q_i m_e)/(q_e m_i) (Sec. 2.6)
    fac = (QE * ME) / (-QE * MAR)
    np.testing.assert_allclose(ions["az"], 0.5 * a0[1] * fac, rtol=1e-12)


def test_collisions_conserve_energy_up_to_thresholds():
    """Elastic collisions lose 2(m/M)(1 - cos chi) E, excitation loses its threshold,
    ionisation shares E - thr between two electrons (Sec. 2.6)."""
    cfg = W.config("c1", split_every=0)
    o = Oracle(cfg, capacity=400_000)
    N = 100_000
    E = 90.0
    v = np.sqrt(2 * E * QE / ME)
    o.set_particles(0, _state(N, vz=v))
    o.set_particles(1, _state(0))
    _zero_fields(o)
    o.particle_pass()  # E = 0, a = 0: the first push keeps every speed
    e = o.get_particles(0)
    Etot = (0.5 * ME * (e["vr"] ** 2 + e["vt"] ** 2 + e["vz"] ** 2) / QE).sum()
    c, _ = o.counters()
    n_el, n_ex, n_iz = c[C_COLL], c[C_COLL + 1], c[C_COLL + 2]
    assert n_iz > 100 and n_ex > 100
    expect = N * E - n_ex * 11.5 - n_iz * 15.76
    assert expect - n_el * E * 4 * ME / MAR - 1e-6 * N * E <= Etot <= expect + 1e-6 * N * E


def test_split_conserves_weight_and_momentum():
    cfg = W.config("c1", split_every=1)
    cfg["gas"] = dict(cfg["gas"], p_Pa=0.0)
    o = Oracle(cfg, capacity=2_000_000)
    rng = np.random.default_rng(2)
    N = 3000
    st = W.random_particles(cfg, 0, N, seed=8, margin=0.003)
    st["r"] = np.minimum(st["r"], cfg["R"] - 0.003)
    # weights up to ~30 reference weights
    j = np.floor(st["r"] / (cfg["R"] / (cfg["nr"] - 1))).astype(int)
    wr = np.array([o.w_ref(0, int(k)) for k in j])
    st["w"] = wr * rng.uniform(0.2, 30.0, N)
    st["vr"] *= 1e-6
    st["vt"] *= 1e-6
    st["vz"] *= 1e-6
    o.set_particles(0, st)
    o.set_particles(1, _state(0))
    _zero_fields(o)
    W0 = st["w"].sum()
    P0 = np.array([(st["w"] * st[k]).sum() for k in ("vr", "vt", "vz")])
    o.particle_pass()
    p = o.get_particles(0)
    assert abs(p["w"].sum() / W0 - 1) < 1e-13
    # momentum: the first push rotates v_r, v_theta; compare |w v_z| sums and speeds
    assert abs((p["w"] * p["vz"]).sum() / P0[2] - 1) < 1e-12
    c, _ = o.counters()
    n_split = int((st["w"] > wr).sum())
    assert c[C_SPLITS] == n_split
    expect_new = 0
    for w, r in zip(st["w"], wr):
        if w > r:
            k = int(np.floor(w / r))
            expect_new += k if w - k * r > 0 else k - 1
    assert len(p["w"]) == N + expect_new
    # every particle now carries at most one reference weight (to rounding)
    jj = np.floor(p["r"] / (cfg["R"] / (cfg["nr"] - 1))).astype(int)
    wr2 = np.array([o.w_ref(0, int(k)) for k in jj])
    assert np.all(p["w"] <= wr2 * (1 + 1e-9))


def test_reference_weight_equals_load_weight():
    cfg = W.scaled(W.config("c1"), 2048 * 3)  # exactly 3 per cell
    o = Oracle(cfg)
    o.load()
    p = o.get_particles(0)
    dr = cfg["R"] / (cfg["nr"] - 1)
    j = np.floor(p["r"] / dr).astype(int)
    wr = np.array([o.w_ref(0, int(k)) for k in j])
    np.testing.assert_allclose(p["w"], wr, rtol=1e-14)


def test_step_conserves_charge_and_particles():
    cfg = W.scaled(W.config("c1"), 20_000)
    o = Oracle(cfg)
    o.load()
    q = [sp["q"] for sp in cfg["species"]]
    Q0 = sum(q[s] * o.get_particles(s)["w"].sum() for s in (0, 1))
    n0 = [o.count(0), o.count(1)]
    o.step(5)
    c, qa = o.counters()
    Q1 = sum(q[s] * o.get_particles(s)["w"].sum() for s in (0, 1))
    # the charge that left through the walls plus what is inside is conserved
    assert abs((Q1 + qa.sum()) - Q0) < 1e-9 * abs(q[0] * o.get_particles(0)["w"].sum())
    for s in (0, 1):
        absorbed = c[C_ABS + 3 * s: C_ABS + 3 * s + 3].sum()
        assert o.count(s) == n0[s] - absorbed + c[C_BIRTHS + s]


def test_implicit_step_is_stable_at_large_plasma_frequency_times_dt():
    """The D1 scheme with the implicit susceptibility stays bounded at w_p dt >> 2, where an
    explicit leapfrog diverges (Sec. 1 and 2.1)."""
    cfg = W.config("c1", nz=33, nr=17, R=0.01, L=0.02, split_every=0, mg_tol=1e-12)
    cfg["gas"] = dict(cfg["gas"], p_Pa=0.0)
    cfg["rf"] = dict(amp=[0.0], freq=[0.0], phase=[0.0])
    n0 = 2e17  # w_p = 2.5e10 /s, w_p dt = 4.6
    for sp in cfg["species"]:
        sp["n0"] = n0
        sp["T_eV"] = 1e-3
    cfg = W.scaled(cfg, 40 * 32 * 16)
    wp = np.sqrt(n0 * QE ** 2 / (8.8541878128e-12 * ME))
    assert wp * cfg["dt"] > 4
    o = Oracle(cfg)
    o.load()
    # electron displacement: z -> z + d sin(pi z / L)
    e = o.get_particles(0)
    e["z"] = e["z"] + 2e-5 * np.sin(np.pi * e["z"] / cfg["L"])
    o.set_particles(0, e)
    energy = []
    for _ in range(40):
        o.step(1)
        Ez = o.grid("Ez")
        energy.append((Ez[1:-1, :-1] ** 2).sum())
    energy = np.array(energy)
    assert np.all(np.isfinite(energy))
    assert energy[-10:].max() < 2.0 * energy[:5].max()
