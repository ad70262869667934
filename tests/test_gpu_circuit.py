"""External circuit on the CUDA path (Sec. 2.5, end: blocking capacitor by
Vahedi's superposition) against the FP64 oracle, through the C ABI.

The step solves twice (phi_P with the plasma's charge and the electrode at
0, phi_L charge-free with the electrode at 1), takes the electrode voltage
from the circuit equation and superposes.  FP64: 1e-11 relative over several
steps, like the multi-step parity of the directly driven reactor; mixed:
the electrode voltage to 1e-6 of the source amplitude.
"""
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


def _cfg(prec, C, n=20_000):
    cfg = W.scaled(W.config("c1", precision=prec), n)
    cfg["circuit_C"] = C
    return cfg


def _amp(cfg):
    return sum(abs(a) for a in cfg["rf"]["amp"])


def test_circuit_multi_step_parity_fp64(pic):
    cfg = _cfg("fp64", 1e-10)
    o = Oracle(cfg)
    o.load()
    h = pic.pic_init(cfg)
    for _ in range(4):
        pic.pic_step(h, 2)
        o.step(2)
        Vg, Qg, Qcg = pic.pic_get_circuit(h)
        Vo, Qo, Qco = o.circuit()
        assert abs(Vg - Vo) <= 1e-11 * _amp(cfg), (Vg, Vo)
        assert abs(Qg - Qo) <= 1e-11 * max(abs(Qo), abs(Qco)), (Qg, Qo)
        assert abs(Qcg - Qco) <= 1e-11 * max(abs(Qo), abs(Qco)), (Qcg, Qco)
    o.finalize()
    f = pic.pic_get_fields(h)
    for name in ("phi", "Ez", "Er"):
        assert nerr(f[name], o.grid(name)) < 1e-11, name
    assert np.allclose(f["phi"][0, :-1], Vg, rtol=0, atol=1e-12 * _amp(cfg))
    emax = P.e_max({k: o.grid(k) for k in ("Ez", "Er")})
    for s in (0, 1):
        g, ref = by_id(pic.pic_get_particles(h, s)), by_id(o.get_particles(s))
        assert np.array_equal(g["id"], ref["id"])
        # element by element over eight steps (tests/parity.py)
        e = P.errors(cfg, s, g, ref, emax, P.w_ref_table(cfg, s))
        assert e.max() < 1e-10, (s, float(e.max()))
    # the capacitor has started to charge: the electrode is off the source
    t = o.step_index() * o.cfg["dt"]
    assert Qcg != 0.0 and abs(Vg - o.voltage(t)) > 0.0


def test_circuit_parity_mixed(pic):
    cfg = _cfg("mixed", 1e-10)
    o = Oracle(cfg)
    o.load()
    h = pic.pic_init(cfg)
    pic.pic_step(h, 3)
    o.step(3)
    Vg, Qg, Qcg = pic.pic_get_circuit(h)
    Vo, Qo, Qco = o.circuit()
    assert abs(Vg - Vo) <= 1e-6 * _amp(cfg), (Vg, Vo)
    o.finalize()
    f = pic.pic_get_fields(h)
    assert nerr(f["phi"], o.grid("phi")) < 1e-5


def test_large_capacitor_is_direct_drive(pic):
    """C -> infinity on the GPU: the superposed field is the directly driven one."""
    a = pic.pic_init(_cfg("fp64", 0.0))
    b = pic.pic_init(_cfg("fp64", 1e3))
    pic.pic_step(a, 4)
    pic.pic_step(b, 4)
    pa, pb = pic.pic_get_fields(a)["phi"], pic.pic_get_fields(b)["phi"]
    assert nerr(pb, pa) < 1e-9
    V, _, _ = pic.pic_get_circuit(b)
    assert np.allclose(pb[0, :-1], V, rtol=0, atol=1e-12 * 100.0)


def test_circuit_checkpoint_resume(pic, tmp_path):
    cfg = _cfg("fp64", 1e-10)
    h1 = pic.pic_init(cfg)
    pic.pic_step(h1, 3)
    path = str(tmp_path / "ck_circuit.bin")
    pic.pic_save(h1, path)
    h2 = pic.pic_init(cfg, load=False)
    pic.pic_load(h2, path)
    assert pic.pic_get_circuit(h2) == pic.pic_get_circuit(h1)
    pic.pic_step(h1, 2)
    pic.pic_step(h2, 2)
    c1, c2 = pic.pic_get_circuit(h1), pic.pic_get_circuit(h2)
    assert abs(c1[0] - c2[0]) <= 1e-12 * 100.0
    fa, fb = pic.pic_get_fields(h1), pic.pic_get_fields(h2)
    assert nerr(fb["phi"], fa["phi"]) < 1e-12
    for s in (0, 1):
        a, b = by_id(pic.pic_get_particles(h1, s)), by_id(pic.pic_get_particles(h2, s))
        assert np.array_equal(a["id"], b["id"])
        for k in FIELDS:
            assert nerr(b[k], a[k]) < 1e-12, k
    # a checkpoint of a circuit run does not load into a directly driven reactor
    h3 = pic.pic_init(_cfg("fp64", 0.0), load=False)
    with pytest.raises(pic.PicError):
        pic.pic_load(h3, path)


def test_negative_circuit_capacitance_is_rejected(pic):
    with pytest.raises(pic.PicError):
        pic.pic_init(_cfg("fp64", -1.0))
