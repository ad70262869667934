"""Pins of the oracle's external circuit (Sec. 2.5, end: blocking capacitor by
Vahedi's superposition)."""
import numpy as np

import workloads as W
from oracle import Oracle


def _cfg(C, n=20_000):
    cfg = W.scaled(W.config("c1"), n)
    cfg["circuit_C"] = C
    return cfg


def test_large_capacitor_is_direct_drive():
    """C -> infinity: the capacitor holds no voltage, V = V_rf, and the
    superposition phi_P + V phi_L is the directly driven solution."""
    a, b = Oracle(_cfg(0.0)), Oracle(_cfg(1e3))
    for o in (a, b):
        o.load()
        o.step(5)
        o.finalize()
    pa, pb = a.grid("phi"), b.grid("phi")
    assert np.abs(pa - pb).max() <= 1e-9 * np.abs(pa).max()
    V, Q, Qc = b.circuit()
    t = (b.step_index()) * b.cfg["dt"]
    assert abs(V - b.voltage(t)) <= 1e-9 * 100.0
    assert np.allclose(pb[0, :-1], V, rtol=0, atol=1e-12 * 100.0)


def test_circuit_equation_holds_step_by_step():
    """Q^t - Q^{t-1} = (Q_c^t - Q_c^{t-1}) + Q_conv^t, Q_conv^t the charge the
    electrode collected in the previous step's particle pass; V = V_rf - Q_c/C;
    the electrode row of phi sits at V."""
    C = 1e-10
    o = Oracle(_cfg(C))
    o.load()
    prev = (0.0, 0.0)  # Q, Q_c before the first step
    q_before = [0.0, 0.0]  # collected charge at z = 0 before the last two passes
    for k in range(12):
        o.step(1)
        V, Q, Qc = o.circuit()
        q_conv = q_before[1] - q_before[0]
        assert abs((Q - prev[0]) - (Qc - prev[1]) - q_conv) <= 1e-12 * max(abs(Q), abs(Qc), 1e-12)
        t = o.step_index() * o.cfg["dt"]
        assert abs(V - (o.voltage(t) - Qc / C)) <= 1e-9 * 100.0
        assert np.allclose(o.grid("phi")[0, :-1], V, rtol=0, atol=1e-12 * 100.0)
        prev = (Q, Qc)
        q_before = [q_before[1], o.counters()[1][0]]


def test_self_bias_is_negative():
    """Electrons reach the electrode faster than ions: the capacitor charges
    so that the electrode sits below the source (Q_c = C (V_rf - V) > 0)."""
    o = Oracle(_cfg(1e-10))
    o.load()
    o.step(200)
    V, Q, Qc = o.circuit()
    assert Qc > 0.0
    assert V < o.voltage(o.step_index() * o.cfg["dt"])
