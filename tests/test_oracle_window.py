"""Pins of the oracle's collisionless window and of its autograd gradient
(the reference for the CUDA path's hand-written adjoint).

The window forward (PyTorch, exact field solve) is pinned to the C oracle's
timestep with the cross sections set to zero; the gradient is pinned to
central finite differences of that forward and to charge conservation (a
uniform weight makes J independent of the parameters).
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle

torch = pytest.importorskip("torch")
from oracle.window import Window, window_J, window_grad  # noqa: E402


def small_cfg(nz=17, nr=33, n0=1e14):
    cfg = W.collisionless(W.config("c1"))
    cfg.update(nz=nz, nr=nr)
    for sp in cfg["species"]:
        sp["n0"] = n0
    return cfg


def small_parts(cfg, n=3000, seed=1):
    vol = np.pi * cfg["R"] ** 2 * cfg["L"]
    ws = cfg["species"][0]["n0"] * vol / n
    e = W.random_particles(cfg, 0, n, seed=seed, hot=1.0, accel=1e14, wscale=ws, margin=1e-4)
    i = W.random_particles(cfg, 1, n, seed=seed + 1, hot=3.0, accel=1e9, wscale=ws, margin=1e-4)
    return [e, i]


def weight(cfg):
    return W.gaussian_weight(cfg, centre=(0.02, 0.01), sigma=0.005)


def test_window_forward_matches_the_oracle_timestep():
    cfg = small_cfg()
    parts = small_parts(cfg)
    K, step0 = 8, 5
    w = weight(cfg)
    o = Oracle(cfg)
    for s in (0, 1):
        o.set_particles(s, parts[s])
    o.set_step(step0)
    o.deposit()
    o.reset_moments()
    o.step(K)
    V = Window(cfg).V.numpy()
    J_c = float((w * V * o.moments()["ni"]).sum())
    trace = []
    J_t = window_J(cfg, parts, w, K, step0=step0, trace=trace)
    assert abs(J_t - J_c) <= 1e-9 * abs(J_c)
    # final states, alive particles matched by id
    st = trace[-1]["st"]
    for s in (0, 1):
        ref = o.get_particles(s)
        alive = st[s][7].numpy()
        ids = np.asarray(parts[s]["id"])[alive]
        assert np.array_equal(np.sort(ids), np.sort(ref["id"]))
        oi = np.argsort(ref["id"])
        ti = np.argsort(ids)
        for k, name in enumerate(("r", "z", "vr", "vt", "vz", "ar", "az")):
            a = st[s][k].numpy()[alive][ti]
            b = ref[name][oi]
            assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max(), (s, name)
    # some electrons reached a wall, so the alive bookkeeping was exercised
    assert (~st[0][7].numpy()).sum() > 0


def test_window_gradient_matches_central_differences():
    cfg = small_cfg()
    parts = small_parts(cfg, n=2000, seed=7)
    K = 6
    w = weight(cfg)
    J, dA, dP = window_grad(cfg, parts, w, K)
    # J moves by ~1e-11 of itself per volt (ions barely move in K steps), so
    # the differences lose ~5 digits to cancellation; steps of a few volts
    # (amplitude) and 0.1 V (one boundary node) keep both errors near 1e-5
    amp = cfg["rf"]["amp"][0]
    h = 3e-2 * amp
    fd = (window_J(cfg, parts, w, K, amp0=amp + h) - window_J(cfg, parts, w, K, amp0=amp - h)) / (2 * h)
    assert abs(fd - dA) <= 1e-4 * abs(dA) + 1e-12 * abs(J), (fd, dA)
    scale = np.abs(dP).max()
    assert scale > 0
    for j in (0, 7, 16, 30):
        pz = np.zeros(cfg["nr"])
        pz[j] = 0.1
        fd = (window_J(cfg, parts, w, K, phi_zL=pz) - window_J(cfg, parts, w, K, phi_zL=-pz)) / 0.2
        assert abs(fd - dP[j]) <= 1e-4 * scale, (j, fd, dP[j])


def test_uniform_weight_makes_the_gradient_vanish():
    """With w = 1 the functional is the ions' total weight (the shape factors
    sum to one), independent of the field: charge conservation of the deposit
    carries through the adjoint."""
    cfg = small_cfg()
    parts = small_parts(cfg, n=1500, seed=11)
    K = 5
    J1, dA1, dP1 = window_grad(cfg, parts, np.ones((cfg["nz"], cfg["nr"])), K)
    assert abs(J1 - parts[1]["w"].sum()) <= 1e-12 * J1   # no ion reached a wall
    _, dA, dP = window_grad(cfg, parts, weight(cfg), K)
    assert abs(dA1) <= 1e-9 * abs(dA)
    assert np.abs(dP1).max() <= 1e-9 * np.abs(dP).max()


def test_tiny_mesh_full_steps_against_the_dense_forward():
    """Brute force on the smallest case: 8 particles per species on the 5 x 5
    mesh, several full (collisionless) steps of the oracle against the window
    forward written out with a dense solve of the field."""
    cfg = W.collisionless(W.config("tiny"))
    parts = [W.random_particles(cfg, s, 8, seed=50 + s, hot=1.0 + 9.0 * s, margin=2e-4) for s in (0, 1)]
    K, step0 = 4, 2
    w = np.ones((cfg["nz"], cfg["nr"]))
    o = Oracle(cfg)
    for s in (0, 1):
        o.set_particles(s, parts[s])
    o.set_step(step0)
    o.deposit()
    o.reset_moments()
    o.step(K)
    trace = []
    J_t = window_J(cfg, parts, w, K, step0=step0, trace=trace)
    V = Window(cfg).V.numpy()
    assert abs(J_t - float((w * V * o.moments()["ni"]).sum())) <= 1e-12 * abs(J_t)
    o.finalize()
    assert np.abs(trace[-1]["phi"].numpy() - o.grid("phi")).max() <= 1e-9 * np.abs(o.grid("phi")).max()
    for s in (0, 1):
        ref = o.get_particles(s)
        st = trace[-1]["st"][s]
        alive = st[7].numpy()
        ids = np.asarray(parts[s]["id"])[alive]
        assert np.array_equal(np.sort(ids), np.sort(ref["id"]))
        oi, ti = np.argsort(ref["id"]), np.argsort(ids)
        for k, name in enumerate(("r", "z", "vr", "vt", "vz", "ar", "az")):
            a, b = st[k].numpy()[alive][ti], ref[name][oi]
            assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1e-300), (s, name)
