"""The element-wise comparison used by the GPU parity tests (tests/parity.py),
checked on the CPU against the oracle alone.

The mixed path may take an integer decision differently from the FP64 oracle
only where a value sits within FP32 rounding of the threshold.  The helper's
explain() must accept such a case and reject a state that no rounding-sized
perturbation of the inputs reaches.  The case built here is the split
threshold (Sec. 2.2): a weight a hair above 3 w_r splits into 3 copies in
FP64 and into 2 after one FP32 rounding down.
"""
import numpy as np

import parity as P
import workloads as W
from oracle import Oracle


def _setup():
    cfg = W.collisionless(W.config("c1"))
    cfg["split_every"] = 1
    cfg["species"] = [dict(sp, n_init=0, capacity=4096) for sp in cfg["species"]]
    dr = cfg["R"] / (cfg["nr"] - 1)
    o = Oracle(cfg, capacity=64)
    r = 10.5 * dr
    wr = o.w_ref(0, 10)
    inp = dict(r=np.array([r]), z=np.array([0.01]), vr=np.array([1e4]), vt=np.array([0.0]),
               vz=np.array([2e4]), ar=np.zeros(1), az=np.zeros(1), w=np.array([3.0 * wr * (1 + 1e-8)]),
               id=np.array([7], dtype=np.uint64))
    grids = {"Ez": np.full((cfg["nz"], cfg["nr"]), 10.0), "Er": np.zeros((cfg["nz"], cfg["nr"]))}
    return cfg, inp, grids, wr


def _pass(cfg, inp, grids):
    o = Oracle(cfg, capacity=4096)
    o.set_grid("Ez", grids["Ez"])
    o.set_grid("Er", grids["Er"])
    o.set_step(0)
    o.set_particles(0, inp)
    o.set_next_id(0, 1000)
    o.set_next_id(1, 1000)
    o.particle_pass()
    out = o.get_particles(0)
    k = int(np.nonzero(out["id"] == 7)[0][0])
    return {f: out[f][k:k + 1] for f in out}, len(out["id"])


def test_explain_accepts_a_split_decision_within_fp32_rounding():
    cfg, inp, grids, wr = _setup()
    exact, n_exact = _pass(cfg, inp, grids)
    rounded = dict(inp, w=inp["w"] * (1.0 - 2.0 ** -23))
    flipped, n_flipped = _pass(cfg, rounded, grids)
    assert n_exact == 4 and n_flipped == 3  # 3 copies + parent, against 2 + parent
    assert exact["w"][0] < 1e-6 * wr and abs(flipped["w"][0] - wr) < 1e-6 * wr
    assert P.explain(cfg, 0, 7, inp, grids, 0, flipped, "mixed")


def test_explain_rejects_a_state_no_rounding_reaches():
    cfg, inp, grids, wr = _setup()
    exact, _ = _pass(cfg, inp, grids)
    wrong = dict(exact, w=exact["w"] + 0.5 * wr)
    assert not P.explain(cfg, 0, 7, inp, grids, 0, wrong, "mixed", tries=16)
    moved = dict(exact, vz=exact["vz"] * (1 + 1e-3))
    assert not P.explain(cfg, 0, 7, inp, grids, 0, moved, "mixed", tries=16)


def test_check_sorted_rejects_repeats_and_disorder():
    ok = dict(cell=np.array([0, 0, 3, 5]), id=np.array([4, 1, 2, 3], dtype=np.uint64))
    P.check_sorted(ok, 8)
    for bad in (dict(ok, cell=np.array([0, 3, 0, 5])), dict(ok, id=np.array([4, 1, 4, 3], dtype=np.uint64)),
                dict(ok, cell=np.array([0, 0, 3, 8]))):
        try:
            P.check_sorted(bad, 8)
        except AssertionError:
            continue
        raise AssertionError("check_sorted accepted a bad permutation")
