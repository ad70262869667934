"""Long runs: the GPU path against the FP64 oracle statistically.

After a few hundred steps two runs from the same start differ (deposit
atomics add in any order, FP32 rounding in the mixed path, and the motion
is chaotic), so time averages are compared: density and potential
(volume-weighted over 2 x 4 regions of the mesh), the mean electron energy and
the EEDF in energy bands.  Each statistic of the GPU run (seed 1) must lie
within 1 % of the oracle's seed-1 value, or within 3 sigma, where sigma is
the seed-to-seed spread of that statistic over K independent oracle runs
(the difference of two runs carries sqrt(2) sigma).  Workload: the small
reactor (33 x 65 nodes, 1e5 electrons + 1e5 ions), 200 steps, averages over
the last 100.
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle

pytestmark = pytest.mark.gpu

STEPS, AVG, K = 200, 100, 6


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic as P

    build()
    return P


def _regions(a, w, nz, nr, bz=2, br=4):
    """Weighted sums of a over blocks of nodes (bz rows x br columns), and the weights."""
    iz = np.minimum(np.arange(nz) * bz // nz, bz - 1)
    jr = np.minimum(np.arange(nr) * br // nr, br - 1)
    s = np.zeros((bz, br))
    ws = np.zeros((bz, br))
    np.add.at(s, (iz[:, None], jr[None, :]), a * w)
    np.add.at(ws, (iz[:, None], jr[None, :]), w)
    return s, ws


def stats(cfg, m, V):
    """The compared statistics of one run, with the scale its 1 % refers to."""
    nz, nr = cfg["nz"], cfg["nr"]
    out = {}
    for key in ("ne", "ni"):
        s, _ = _regions(m[key], V, nz, nr)  # charge carriers per region
        big = s / s.sum() > 0.01
        out[key] = (s[big], np.abs(s[big]))
    s, ws = _regions(m["phi"], V, nz, nr)
    phi = s / ws
    out["phi"] = (phi.ravel(), np.full(phi.size, np.abs(m["phi"]).max()))
    e = (np.arange(cfg["eedf_bins"]) + 0.5) * cfg["eedf_emax"] / cfg["eedf_bins"]
    f = m["eedf"] / m["eedf"].sum()
    mean = (e * f).sum()
    out["mean_energy"] = (np.array([mean]), np.array([mean]))
    bands = [0, 2, 5, 10, 20, 100]
    fr = np.array([f[(e >= a) & (e < b)].sum() for a, b in zip(bands[:-1], bands[1:])])
    out["eedf_bands"] = (fr, fr)
    return out


def _oracle(seed):
    cfg = W.config("c1", seed=seed)
    o = Oracle(cfg)
    o.load()
    o.step(STEPS - AVG)
    o.reset_moments()
    o.step(AVG)
    m = o.moments()
    return cfg, m, o.node_volumes()


@pytest.fixture(scope="module")
def oracle_runs():
    runs = [_oracle(1 + k) for k in range(K)]
    cfg, m1, V = runs[0]
    st = [stats(cfg, m, V) for _, m, _ in runs]
    sigma = {key: np.std(np.array([s[key][0] for s in st]), axis=0, ddof=1) for key in st[0]}
    return cfg, m1, V, st[0], sigma


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_time_averages_match_the_oracle(pic, oracle_runs, prec):
    cfg, om, V, ost, sigma = oracle_runs
    h = pic.pic_init(W.config("c1", precision=prec))
    assert pic.pic_step(h, STEPS - AVG) == 0
    pic.pic_moments(h, reset=True)
    assert pic.pic_step(h, AVG) == 0
    gm = pic.pic_moments(h)
    assert gm["nsamples"] == om["nsamples"] == AVG
    gst = stats(cfg, gm, V)
    for key, (o, scale) in ost.items():
        g = gst[key][0]
        assert g.shape == o.shape, key
        lim = np.maximum(0.01 * scale, 3.0 * np.sqrt(2.0) * sigma[key])
        worst = np.max(np.abs(g - o) / lim)
        assert worst <= 1.0, (key, worst, g, o)
