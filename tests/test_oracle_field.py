"""Pins of the oracle's field solver (Sec. 2.5): operator properties, a dense direct
solve, a manufactured solution with second-order convergence, the paper's multigrid
convergence claims, and the E-field differences."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import Oracle

HERE = os.path.dirname(os.path.abspath(__file__))
EPS0 = 8.8541878128e-12


def _golden_mg():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_mg_convergence.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _cfg(nz, nr, R=0.05, L=0.02, **kw):
    return W.config("c1", nz=nz, nr=nr, R=R, L=L, **kw)


def _interior_mask(nz, nr):
    m = np.zeros((nz, nr), bool)
    m[1:-1, :-1] = True
    return m


@pytest.mark.parametrize("face", ["max", "mean"])
def test_operator_symmetric_and_rows_sum_to_zero(face):
    cfg = _cfg(9, 13, chi_face=face)
    o = Oracle(cfg)
    chi = W.random_grid(cfg, seed=3, scale=2.0, smooth=False)
    rng = np.random.default_rng(0)
    mask = _interior_mask(9, 13)
    u = np.where(mask, rng.normal(size=(9, 13)), 0.0)
    v = np.where(mask, rng.normal(size=(9, 13)), 0.0)
    Au, Av = o.apply_A(chi, u), o.apply_A(chi, v)
    assert abs((v * Au).sum() - (u * Av).sum()) < 1e-12 * np.abs(v * Au).sum()
    # b = a + c + d + e: a constant is in the kernel of every interior row
    one = o.apply_A(chi, np.ones((9, 13)))
    assert np.abs(one[mask]).max() < 1e-12 * np.abs(Au).max()
    # positive definite on the interior unknowns
    assert (u * Au).sum() > 0


def _dense_solve(o, chi, rho, V, phiL=None):
    nz, nr = o.nz, o.nr
    mask = _interior_mask(nz, nr)
    idx = np.flatnonzero(mask)
    n = len(idx)
    A = np.zeros((n, n))
    for k, p in enumerate(idx):
        e = np.zeros(nz * nr)
        e[p] = 1.0
        A[:, k] = o.apply_A(chi, e.reshape(nz, nr)).reshape(-1)[idx]
    ubc = np.zeros((nz, nr))
    ubc[0, :-1] = V
    if phiL is not None:
        ubc[-1, :] = phiL
    f = o.rhs(rho).reshape(-1)[idx] - o.apply_A(chi, ubc).reshape(-1)[idx]
    x = np.linalg.solve(A, f)
    out = ubc.copy().reshape(-1)
    out[idx] = x
    return out.reshape(nz, nr)


@pytest.mark.parametrize("face", ["max", "mean"])
def test_multigrid_equals_dense_direct_solve(face):
    cfg = _cfg(9, 17, chi_face=face)
    o = Oracle(cfg)
    chi = W.random_grid(cfg, seed=5, scale=3.0)
    rho = 1e-6 * (W.random_grid(cfg, seed=6, smooth=False) - 0.5)
    o.set_grid("chi", chi)
    o.set_grid("rho", rho)
    o.set_grid("phi", np.zeros((9, 17)))
    st, cyc, res = o.solve(37.0, tol=1e-14, max_cycles=200)
    assert st == 0 and res <= 1e-14
    ref = _dense_solve(o, chi, rho, 37.0)
    np.testing.assert_allclose(o.grid("phi"), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def _manufactured(R, L):
    sp = pytest.importorskip("sympy")
    r, z = sp.symbols("r z", nonnegative=True)
    phi = (sp.cos(sp.pi * r / (2 * R)) * sp.sin(sp.pi * z / L)
           + sp.Rational(3, 10) * (1 - r ** 2 / R ** 2) * sp.sin(2 * sp.pi * z / L)
           + sp.Rational(1, 2) * (z / L) * sp.cos(sp.pi * r / (2 * R)))
    chi = 1 + sp.Rational(1, 2) * sp.cos(sp.pi * r / R) * sp.sin(sp.pi * z / L)
    eps = 1 + chi
    div = sp.diff(r * eps * sp.diff(phi, r), r) / r + sp.diff(eps * sp.diff(phi, z), z)
    rho = -EPS0 * div
    f_phi = sp.lambdify((r, z), phi, "numpy")
    f_chi = sp.lambdify((r, z), chi, "numpy")
    f_rho = sp.lambdify((r, z), rho, "numpy")
    return f_phi, f_chi, f_rho


def test_manufactured_solution_second_order():
    """Smooth eps = 1 + chi(r, z), phi even in r, Dirichlet data on z = 0, z = L, r = R:
    the FV scheme with the mean face rule converges at second order (Sec. 2.5)."""
    R, L = 0.05, 0.02
    f_phi, f_chi, f_rho = _manufactured(R, L)
    errs = []
    for nz, nr in ((9, 17), (17, 33), (33, 65), (65, 129)):
        cfg = _cfg(nz, nr, R=R, L=L, chi_face="mean")
        zz = np.linspace(0, L, nz)[:, None] * np.ones((1, nr))
        rr = np.ones((nz, 1)) * np.linspace(0, R, nr)[None, :]
        rsafe = np.where(rr == 0, 1e-12 * R, rr)
        ex = f_phi(rr, zz)
        cfg["phi_zL"] = ex[-1, :].copy()
        o = Oracle(cfg)
        o.set_grid("chi", f_chi(rr, zz) * np.ones((nz, nr)))
        o.set_grid("rho", f_rho(rsafe, zz))
        o.set_grid("phi", np.zeros((nz, nr)))
        st, cyc, res = o.solve(0.0, tol=1e-13, max_cycles=300)
        assert st == 0
        errs.append(np.abs(o.grid("phi") - ex).max())
    ratios = [errs[k] / errs[k + 1] for k in range(len(errs) - 1)]
    assert all(3.5 < q < 4.6 for q in ratios[1:]), (errs, ratios)


def test_max_face_rule_still_converges():
    R, L = 0.05, 0.02
    f_phi, f_chi, f_rho = _manufactured(R, L)
    errs = []
    for nz, nr in ((17, 33), (33, 65), (65, 129)):
        cfg = _cfg(nz, nr, R=R, L=L, chi_face="max")
        zz = np.linspace(0, L, nz)[:, None] * np.ones((1, nr))
        rr = np.ones((nz, 1)) * np.linspace(0, R, nr)[None, :]
        ex = f_phi(rr, zz)
        cfg["phi_zL"] = ex[-1, :].copy()
        o = Oracle(cfg)
        o.set_grid("chi", f_chi(rr, zz) * np.ones((nz, nr)))
        o.set_grid("rho", f_rho(np.where(rr == 0, 1e-12 * R, rr), zz))
        o.set_grid("phi", np.zeros((nz, nr)))
        assert o.solve(0.0, tol=1e-13, max_cycles=300)[0] == 0
        errs.append(np.abs(o.grid("phi") - ex).max())
    # max(chi_i, chi_{i+1}) differs from the face value by O(h |grad chi|): first order
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r1 > 1.5 and r2 > r1 and r2 < 2.2, errs


def _cycles(nz, nr, chi_value, tol, R=0.05, L=0.02, seed=9):
    cfg = _cfg(nz, nr, R=R, L=L)
    o = Oracle(cfg)
    zz = np.linspace(0, 1, nz)[:, None]
    rr = np.linspace(0, 1, nr)[None, :]
    chi = chi_value * (1 + 0.5 * np.cos(np.pi * rr) * np.sin(np.pi * zz)) * np.ones((nz, nr))
    if chi_value == 0:
        chi = np.zeros((nz, nr))
    rng = np.random.default_rng(seed)
    rho = 1e-5 * rng.uniform(-1, 1, (nz, nr))
    o.set_grid("chi", chi)
    o.set_grid("rho", rho)
    o.set_grid("phi", np.zeros((nz, nr)))
    st, cyc, res = o.solve(100.0, tol=tol, max_cycles=200)
    assert st == 0
    return cyc


def test_paper_multigrid_convergence_claims():
    g = _golden_mg()
    # chi = 0: the cycle count does not grow with the grid
    c0 = [_cycles(nz, nr, 0.0, 1e-10) for nz, nr in ((17, 33), (33, 65), (65, 129), (129, 257))]
    assert max(c0) - min(c0) <= 2, c0
    # chi ~ 1 smooth: about 12 V-cycles to 1e-10 in the max norm
    c1 = [_cycles(nz, nr, 1.0, g["chi1_tol"]) for nz, nr in ((33, 65), (65, 129), (129, 257))]
    assert all(abs(c - g["chi1_cycles_about"]) <= 4 for c in c1), c1


def test_efield_differences():
    cfg = _cfg(9, 11)
    o = Oracle(cfg)
    L, R = cfg["L"], cfg["R"]
    z = np.linspace(0, L, 9)[:, None]
    r = np.linspace(0, R, 11)[None, :]
    a, b = 1234.0, -5.6e5
    o.set_grid("phi", a * z + b * r * r + 0 * z * r)
    o.efield()
    Ez, Er = o.grid("Ez"), o.grid("Er")
    np.testing.assert_allclose(Ez, -a, rtol=1e-10)  # linear in z: exact everywhere
    np.testing.assert_allclose(Er[:, 1:-1], (-2 * b * r * np.ones((9, 1)))[:, 1:-1], rtol=1e-10)
    assert np.all(Er[:, 0] == 0)  # symmetry axis
    dr = R / 10
    assert np.all(np.abs(Er[:, -1] - (-2 * b * R)) <= abs(b) * dr * 1.0001)  # first order


def _laplace_run(guess, steps):
    """c1 with no particles (no charge, no susceptibility): the potential is
    V(t) times one fixed Laplace solution.  The source is a sine far below its
    first quarter period (2 pi f t < 1e-7 over the run), so V(t_n) is linear in
    n to about 1e-21 of its size."""
    cfg = W.scaled(W.config("c1", precision="fp64", mg_guess=guess, mg_tol=1e-10), 0)
    cfg["rf"] = dict(amp=[1e8], freq=[1.0], phase=[0.0])
    o = Oracle(cfg)
    cyc, phi = [], []
    for _ in range(steps):
        c, _ = o.step(1)
        cyc.append(c)
        phi.append(o.grid("phi"))
    return cfg, o, cyc, phi


def test_linear_start_is_the_next_solution_for_a_voltage_linear_in_time():
    """Algorithm 1's starting value w_0 (Sec. 2.5) taken as 2 phi^n - phi^(n-1):
    for phi(t) = V(t) phi_1 with V linear in t the extrapolated start is the next
    step's solution up to the last two solves' residual errors, so from the third
    step on at most one V-cycle is needed; started from phi^n (the previous
    step's potential) every step needs several.  A sign or index slip in the
    extrapolation (phi^(n-1) - 2 phi^n, or phi^n twice) fails the first claim;
    both starts must reach the same potential within the solve tolerance."""
    steps = 8
    _, _, cyc_lin, phi_lin = _laplace_run("linear", steps)
    _, _, cyc_prev, phi_prev = _laplace_run("previous", steps)
    assert max(cyc_lin[2:]) <= 1, cyc_lin
    assert min(cyc_prev[2:]) >= 4, cyc_prev
    for a, b in zip(phi_lin, phi_prev):
        assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()
    # the potential is V(t) phi_1: each step's is the first one scaled by n
    for n, p in enumerate(phi_prev, start=1):
        assert np.abs(p - n * phi_prev[0]).max() <= 1e-8 * np.abs(p).max()


def test_linear_start_matches_previous_on_the_first_step_and_after_a_set_potential():
    """With no history (a fresh state, or a potential set from outside) the
    extrapolated start is phi^n itself: the first step is bit for bit the one
    started from the previous potential, with the same cycle count."""
    cfg = W.scaled(W.config("c1", precision="fp64"), 2000)
    runs = {}
    for guess in ("linear", "previous"):
        o = Oracle(dict(cfg, mg_guess=guess))
        o.load()
        c1, _ = o.step(1)
        p1 = o.grid("phi")
        o.set_grid("phi", p1)  # no history after this
        c2, _ = o.step(1)
        runs[guess] = (c1, p1, c2, o.grid("phi"))
    a, b = runs["linear"], runs["previous"]
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    assert a[2] == b[2] and np.array_equal(a[3], b[3])
