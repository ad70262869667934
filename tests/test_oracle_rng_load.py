"""Pins of the oracle's Philox generator and of its particle load."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, philox

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert philox(ctr, key) == out


def test_philox_uniformity_chi2():
    # 4096 blocks -> 16384 words, top 6 bits binned: chi^2 with 63 dof
    words = []
    for c in range(4096):
        words += philox([c, 0, 7, 1], [1, 0])
    bins = np.bincount(np.array(words, dtype=np.uint64) >> np.uint64(26), minlength=64)
    e = len(words) / 64
    chi2 = ((bins - e) ** 2 / e).sum()
    assert 30 < chi2 < 110  # ~ p in (1e-3, 1 - 1e-3) for 63 dof


def test_load_cell_counts_and_weights():
    cfg = W.scaled(W.config("c1"), 5000)  # fewer particles than 2048 cells x 3
    o = Oracle(cfg)
    o.load()
    nz, nr, L, R = cfg["nz"], cfg["nr"], cfg["L"], cfg["R"]
    dz, dr = L / (nz - 1), R / (nr - 1)
    for s in (0, 1):
        p = o.get_particles(s)
        assert len(p["r"]) == 5000
        assert np.array_equal(p["id"], np.arange(5000, dtype=np.uint64))
        i = np.floor(p["z"] / dz).astype(int)
        j = np.floor(p["r"] / dr).astype(int)
        c = j * (nz - 1) + i
        ncell = (nz - 1) * (nr - 1)
        counts = np.bincount(c, minlength=ncell)
        base, rem = divmod(5000, ncell)
        expect = np.full(ncell, base)
        expect[:rem] += 1
        assert np.array_equal(counts, expect)
        # the weights of one cell add up to n0 times the cell's volume
        vol = np.pi * ((dr * (j + 1)) ** 2 - (dr * j) ** 2) * dz
        wsum = np.bincount(c, weights=p["w"], minlength=ncell)
        vcell = np.bincount(c, weights=vol, minlength=ncell) / np.maximum(counts, 1)
        n0 = cfg["species"][s]["n0"]
        occ = counts > 0
        np.testing.assert_allclose(wsum[occ], n0 * vcell[occ], rtol=1e-13)
        assert np.all(p["ar"] == 0) and np.all(p["az"] == 0)


def test_load_distributions():
    cfg = W.scaled(W.config("c1"), 200_000)
    o = Oracle(cfg)
    o.load()
    nz, nr, L, R = cfg["nz"], cfg["nr"], cfg["L"], cfg["R"]
    dz, dr = L / (nz - 1), R / (nr - 1)
    for s in (0, 1):
        sp = cfg["species"][s]
        p = o.get_particles(s)
        var = sp["T_eV"] * W.QE / sp["m"]
        for k in ("vr", "vt", "vz"):
            v = p[k]
            assert abs(v.mean()) < 5 * np.sqrt(var / len(v))
            assert abs(v.var() / var - 1) < 5 * np.sqrt(2 / len(v))
        # in-cell offsets: uniform in z and in r^2
        fz = p["z"] / dz - np.floor(p["z"] / dz)
        j = np.floor(p["r"] / dr)
        fr2 = ((p["r"] / dr) ** 2 - j ** 2) / (2 * j + 1)
        for f in (fz, fr2):
            h = np.histogram(f, bins=20, range=(0, 1))[0]
            e = len(f) / 20
            assert ((h - e) ** 2 / e).sum() < 50  # 19 dof


def test_load_range_matches_full_load():
    cfg = W.scaled(W.config("c1"), 20_000)
    o = Oracle(cfg)
    o.load()
    for s in (0, 1):
        full = o.get_particles(s)
        part = o.load_range(s, 1234, 5678)
        for k in full:
            assert np.array_equal(full[k][1234:5678], part[k])
