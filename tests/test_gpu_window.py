"""The collisionless window and its hand-written adjoint on the GPU, through
the C ABI, against the oracle's autograd gradient (oracle/window.py), the
production timestep, finite differences and charge conservation.

Tolerances: the FP64 path's J matches the oracle's exact-solve forward to
1e-9 (the multigrid stops at a relative residual of 1e-10) and its gradient
to 1e-6 of the largest component; the mixed path (FP32 particle states,
FP64 adjoint) to 1e-5 and 1e-3.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic as P

    build()
    return P


def small_cfg(prec, nz=17, nr=33, n0=1e14, n=2000):
    cfg = W.collisionless(W.config("c1", precision=prec))
    cfg.update(nz=nz, nr=nr)
    for sp in cfg["species"]:
        sp["n0"] = n0
        sp["n_init"] = 0
        sp["capacity"] = 4 * n + 4096
    return cfg


def small_parts(cfg, n=2000, seed=7):
    vol = np.pi * cfg["R"] ** 2 * cfg["L"]
    ws = cfg["species"][0]["n0"] * vol / n
    e = W.random_particles(cfg, 0, n, seed=seed, hot=1.0, accel=1e14, wscale=ws, margin=1e-4)
    i = W.random_particles(cfg, 1, n, seed=seed + 1, hot=3.0, accel=1e9, wscale=ws, margin=1e-4)
    return [e, i]


def weight(cfg):
    return W.gaussian_weight(cfg, centre=(0.02, 0.01), sigma=0.005)


def handle(pic, cfg, parts, step0):
    h = pic.pic_init(cfg, load=False)
    for s in (0, 1):
        pic.pic_set_particles(h, s, parts[s])
    pic.pic_set_step(h, step0)
    return h


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_window_gradient_matches_the_oracle(pic, prec):
    from oracle.window import window_grad

    cfg = small_cfg(prec)
    parts = small_parts(cfg)
    K, step0 = 6, 5
    w = weight(cfg)
    Jo, dAo, dPo = window_grad(cfg, parts, w, K, step0=step0)
    h = handle(pic, cfg, parts, step0)
    J, dA, dP = pic.pic_window(h, K, 2, w, cfg["rf"]["amp"][0])
    tj, tg = (1e-9, 1e-6) if prec == "fp64" else (1e-5, 1e-3)
    assert abs(J - Jo) <= tj * abs(Jo), (J, Jo)
    assert abs(dA - dAo) <= tg * abs(dAo), (dA, dAo)
    assert np.abs(dP - dPo).max() <= tg * np.abs(dPo).max(), np.abs(dP - dPo).max() / np.abs(dPo).max()


def test_window_forward_is_the_collisionless_timestep(pic):
    """J of the window equals the functional taken from pic_step's own time
    averages over the same steps (collisionless configuration)."""
    cfg = small_cfg("fp64")
    parts = small_parts(cfg, n=3000, seed=3)
    K, w = 8, weight(cfg)
    h = handle(pic, cfg, parts, 2)
    J, _, _ = pic.pic_window(h, K, 4, w, cfg["rf"]["amp"][0], grad=False)
    pic.pic_moments(h, reset=True)
    pic.pic_step(h, K)
    m = pic.pic_moments(h)
    from oracle.window import Window

    V = Window(cfg).V.numpy()
    Js = float((w * V * m["ni"]).sum())
    assert abs(J - Js) <= 1e-11 * abs(Js), (J, Js)


def test_window_leaves_the_handle_unchanged_and_checkpoints_do_not_matter(pic):
    cfg = small_cfg("fp64")
    parts = small_parts(cfg, n=1500, seed=5)
    h = handle(pic, cfg, parts, 0)
    before = pic.pic_get_particles(h, 0)
    w = weight(cfg)
    out = [pic.pic_window(h, 7, c, w, cfg["rf"]["amp"][0]) for c in (1, 3, 7)]
    after = pic.pic_get_particles(h, 0)
    for k in ("r", "z", "vr", "w", "id"):
        assert np.array_equal(before[k], after[k])
    assert pic.pic_get_counts(h)["step"] == 0
    for J, dA, dP in out[1:]:
        assert abs(J - out[0][0]) <= 1e-12 * abs(out[0][0])
        assert abs(dA - out[0][1]) <= 1e-9 * abs(out[0][1])
        assert np.abs(dP - out[0][2]).max() <= 1e-9 * np.abs(out[0][2]).max()


def test_uniform_weight_gives_a_zero_gradient(pic):
    cfg = small_cfg("fp64")
    parts = small_parts(cfg, n=1500, seed=11)
    h = handle(pic, cfg, parts, 0)
    J1, dA1, dP1 = pic.pic_window(h, 5, 2, np.ones((cfg["nz"], cfg["nr"])), cfg["rf"]["amp"][0])
    assert abs(J1 - parts[1]["w"].sum()) <= 1e-12 * J1
    _, dA, dP = pic.pic_window(h, 5, 2, weight(cfg), cfg["rf"]["amp"][0])
    assert abs(dA1) <= 1e-8 * abs(dA)
    assert np.abs(dP1).max() <= 1e-8 * np.abs(dP).max()


def test_window_autograd_function(pic):
    cfg = small_cfg("fp64")
    parts = small_parts(cfg, n=1000, seed=13)
    h = handle(pic, cfg, parts, 0)
    w = weight(cfg)
    a = torch.tensor(cfg["rf"]["amp"][0], dtype=torch.float64, requires_grad=True)
    p = torch.zeros(cfg["nr"], dtype=torch.float64, requires_grad=True)
    J = pic.window_function().apply(a, p, h, w, 4, 2)
    (3.0 * J).backward()
    # a second call (FP64 atomics add in another order): equal to rounding
    J0, dA, dP = pic.pic_window(h, 4, 2, w, cfg["rf"]["amp"][0])
    assert abs(float(J.detach()) - J0) <= 1e-12 * abs(J0)
    assert abs(float(a.grad) - 3.0 * dA) <= 1e-9 * abs(3.0 * dA)
    assert np.abs(p.grad.numpy() - 3.0 * dP).max() <= 1e-9 * np.abs(3.0 * dP).max()


def test_window_gradient_by_central_differences_c1(pic):
    """c1 mesh, 20k + 20k particles, 10 steps, FP64: the adjoint's dJ/d amp0
    and a few dJ/d phi_zL against central differences of the GPU forward.
    The particles start 3 mm from the walls with cool electrons, so none
    leaves within the window (checked): a particle that reaches a wall makes
    J jump, which a difference quotient sees and a derivative does not."""
    cfg = small_cfg("fp64", nz=33, nr=65, n0=1e15, n=20_000)
    n = 20_000
    vol = np.pi * cfg["R"] ** 2 * cfg["L"]
    ws = 1e15 * vol / n
    parts = [W.random_particles(cfg, 0, n, seed=21, hot=0.3, accel=1e13, wscale=ws, margin=3e-3),
             W.random_particles(cfg, 1, n, seed=22, hot=3.0, accel=1e9, wscale=ws, margin=3e-3)]
    K, amp = 10, cfg["rf"]["amp"][0]
    probe = handle(pic, cfg, parts, 0)
    pic.pic_step(probe, K)
    assert list(pic.pic_get_counts(probe)["n_alive"]) == [n, n]
    h = handle(pic, cfg, parts, 0)
    w = W.gaussian_weight(cfg, centre=(0.02, 0.01), sigma=0.005)
    J, dA, dP = pic.pic_window(h, K, 4, w, amp)
    hA = 0.01 * amp
    fd = (pic.pic_window(h, K, 4, w, amp + hA, grad=False)[0] -
          pic.pic_window(h, K, 4, w, amp - hA, grad=False)[0]) / (2 * hA)
    assert abs(fd - dA) <= 1e-3 * abs(dA), (fd, dA)
    scale = np.abs(dP).max()
    for j in (3, 20, 40):
        pz = np.zeros(cfg["nr"])
        pz[j] = 0.1
        fd = (pic.pic_window(h, K, 4, w, amp, phi_zL=pz, grad=False)[0] -
              pic.pic_window(h, K, 4, w, amp, phi_zL=-pz, grad=False)[0]) / 0.2
        assert abs(fd - dP[j]) <= 1e-3 * scale, (j, fd, dP[j])


def test_window_gradient_by_central_differences_c5_mesh(pic):
    """The adjoint window's mesh (65 x 257) with 1M + 1M particles, FP64,
    8 steps, no particle lost: dJ/d amp0 against central differences of the
    GPU forward.  J moves by ~1e-11 of itself per volt here, so the solves
    run to a relative residual of 1e-13 for the differences to resolve it."""
    cfg = W.collisionless(W.config("c5", precision="fp64", mg_tol=1e-13))
    n = 1_000_000
    for sp in cfg["species"]:
        sp["n_init"] = 0
        sp["capacity"] = n + 4096
        sp["n0"] = 1e13  # weak space charge of the random (not neutral) placement
    vol = np.pi * cfg["R"] ** 2 * cfg["L"]
    ws = cfg["species"][0]["n0"] * vol / n
    parts = [W.random_particles(cfg, 0, n, seed=31, hot=0.2, accel=1e13, wscale=ws, margin=5e-3),
             W.random_particles(cfg, 1, n, seed=32, hot=3.0, accel=1e9, wscale=ws, margin=5e-3)]
    K, amp = 8, cfg["rf"]["amp"][0]
    probe = handle(pic, cfg, parts, 0)
    pic.pic_step(probe, K)
    assert list(pic.pic_get_counts(probe)["n_alive"]) == [n, n]
    h = handle(pic, cfg, parts, 0)
    w = W.gaussian_weight(cfg)
    J, dA, dP = pic.pic_window(h, K, 4, w, amp)
    hA = 0.01 * amp
    fd = (pic.pic_window(h, K, 4, w, amp + hA, grad=False)[0] -
          pic.pic_window(h, K, 4, w, amp - hA, grad=False)[0]) / (2 * hA)
    assert abs(fd - dA) <= 3e-3 * abs(dA), (fd, dA)
