"""Pins of the oracle's particle merging (Sec. 2.2 names it without an
algorithm; the reading is in oracle.c at orc_merge): what a merge of light
particles in pairs must keep and lose, checked against sums taken here,
the pairing rule on a hand-made cell, and the deposit's moments."""
import numpy as np

import workloads as W
from oracle import Oracle


def _sums(cfg, s, p):
    m = cfg["species"][s]["m"]
    w = p["w"]
    return dict(
        w=w.sum(), wz=(w * p["z"]).sum(), wr2=(w * p["r"] ** 2).sum(), pr=(w * p["vr"]).sum(),
        pz=(w * p["vz"]).sum(), L=(w * p["r"] * p["vt"]).sum(), ar=(w * p["ar"]).sum(),
        az=(w * p["az"]).sum(),
        E=0.5 * m * (w * (p["vr"] ** 2 + p["vt"] ** 2 + p["vz"] ** 2)).sum())


def test_merge_keeps_charge_moments_momentum_and_current():
    cfg = W.config("c1")
    for s, dv in ((0, 3e5), (1, 400.0)):
        o = Oracle(cfg)
        o.load()
        before = o.get_particles(s)
        s0 = _sums(cfg, s, before)
        pairs, lost = o.merge(s, 1.5, dv)
        after = o.get_particles(s)
        s1 = _sums(cfg, s, after)
        assert pairs > 1000, pairs
        assert len(after["id"]) == len(before["id"]) - pairs
        assert set(after["id"]).issubset(set(before["id"]))
        w = before["w"]
        scale = dict(w=w.sum(), wz=np.abs(w * before["z"]).sum(), wr2=(w * before["r"] ** 2).sum(),
                     pr=np.abs(w * before["vr"]).sum(), pz=np.abs(w * before["vz"]).sum(),
                     L=np.abs(w * before["r"] * before["vt"]).sum(), ar=np.abs(w * before["ar"]).sum(),
                     az=np.abs(w * before["az"]).sum())
        for k in scale:
            assert abs(s1[k] - s0[k]) <= 1e-12 * max(scale[k], 1e-300), (s, k, s0[k], s1[k])
        # the energy the merge reports is the kinetic energy that went
        assert lost >= 0.0
        assert abs((s0["E"] - s1["E"]) - lost) <= 1e-9 * s0["E"], (s0["E"] - s1["E"], lost)
        # every survivor kept its cell
        dz, dr = cfg["L"] / (cfg["nz"] - 1), cfg["R"] / (cfg["nr"] - 1)
        pos = {int(i): q for q, i in enumerate(before["id"])}
        for q in range(len(after["id"])):
            b = pos[int(after["id"][q])]
            assert int(after["z"][q] // dz) == int(before["z"][b] // dz)
            assert int(after["r"][q] // dr) == int(before["r"][b] // dr)


def test_pairing_rule_on_a_hand_made_cell():
    """One cell: ids 5, 2, 9 light with one velocity bin, id 1 heavy, id 3
    light in another bin.  Ids 2 and 5 merge into 2; 9 stays (odd); 1 and
    3 are untouched."""
    cfg = W.collisionless(W.config("c1"))
    o = Oracle(cfg)
    wr = o.w_ref(0, 10)
    dr, dz = cfg["R"] / (cfg["nr"] - 1), cfg["L"] / (cfg["nz"] - 1)
    ids = np.array([5, 2, 9, 1, 3], dtype=np.uint64)
    z = (7 + np.array([0.1, 0.5, 0.9, 0.3, 0.7])) * dz
    r = (10 + np.array([0.2, 0.8, 0.5, 0.4, 0.6])) * dr
    vr = np.array([1000.0, 1500.0, 1900.0, 1200.0, 9000.0])
    vt = np.array([-300.0, -100.0, -200.0, 0.0, 0.0])
    vz = np.array([50.0, 60.0, 70.0, 0.0, 0.0])
    w = np.array([0.2, 0.3, 0.1, 5.0, 0.2]) * wr
    zero = np.zeros(5)
    o.set_particles(0, dict(r=r, z=z, vr=vr, vt=vt, vz=vz, ar=zero + 1e9, az=zero - 2e9, w=w, id=ids))
    pairs, lost = o.merge(0, 0.5, 2000.0)
    assert pairs == 1
    got = o.get_particles(0)
    assert sorted(int(i) for i in got["id"]) == [1, 2, 3, 9]
    g = {int(i): q for q, i in enumerate(got["id"])}
    a, b = 1, 0  # input positions of ids 2 and 5
    W_ = w[a] + w[b]
    q = g[2]
    assert abs(got["w"][q] - W_) <= 1e-15 * W_
    assert abs(got["z"][q] - (w[a] * z[a] + w[b] * z[b]) / W_) <= 1e-15 * z[a]
    rm = np.sqrt((w[a] * r[a] ** 2 + w[b] * r[b] ** 2) / W_)
    assert abs(got["r"][q] - rm) <= 1e-15 * rm
    assert abs(got["vt"][q] - (w[a] * r[a] * vt[a] + w[b] * r[b] * vt[b]) / (W_ * rm)) <= 1e-12 * 300
    for idx in (1, 3, 9):
        src = int(np.where(ids == idx)[0][0])
        assert got["w"][g[idx]] == w[src] and got["vr"][g[idx]] == vr[src]
    m = cfg["species"][0]["m"]
    # the reported loss is the pair's kinetic energy before less the merged
    # particle's (near the pair's relative kinetic energy; not equal, since
    # v_theta keeps the angular momentum at the merged radius)
    e0 = 0.5 * m * (w[a] * (vr[a] ** 2 + vt[a] ** 2 + vz[a] ** 2) + w[b] * (vr[b] ** 2 + vt[b] ** 2 + vz[b] ** 2))
    e1 = 0.5 * m * W_ * (got["vr"][q] ** 2 + got["vt"][q] ** 2 + got["vz"][q] ** 2)
    assert abs((e0 - e1) - lost) <= 1e-9 * e0
    dvv = np.array([vr[a] - vr[b], vt[a] - vt[b], vz[a] - vz[b]])
    rel = 0.5 * m * w[a] * w[b] / W_ * (dvv @ dvv)
    assert 0.9 * rel < lost < 1.1 * rel


def test_merge_keeps_the_deposits_totals_and_first_moments():
    cfg = W.config("c1")
    o = Oracle(cfg)
    o.load()
    nz, nr = cfg["nz"], cfg["nr"]
    zi = (np.arange(nz) * cfg["L"] / (nz - 1))[:, None]
    rj = (np.arange(nr) * cfg["R"] / (nr - 1))[None, :]
    o.deposit()
    N0 = o.grid("Ne")
    o.merge(0, 1.5, 3e5)
    o.deposit()
    N1 = o.grid("Ne")
    assert np.abs(N1 - N0).max() > 1e-6 * N0.max()  # the deposit did change
    for f in (np.ones_like(zi * rj), zi + 0 * rj, rj ** 2 + 0 * zi):
        m0, m1 = (N0 * f).sum(), (N1 * f).sum()
        assert abs(m1 - m0) <= 1e-12 * abs(m0), (m0, m1)
