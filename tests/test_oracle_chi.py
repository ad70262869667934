"""Pin of the implicit susceptibility's magnitude (Sec. 2.1).

The implicit field equation exists so that the potential solved at step n+1
from the charge deposited at the predicted positions x~ and the
susceptibility chi is, to first order in the particles' final displacement,
the potential of the charge deposited at the final positions x^{n+1}:

    -div(eps0 grad phi^{n+1}) = rho(x^{n+1}) + O(displacement^2).

The final push moves a particle by (1/2)(q/m) E dt^2, so the first-order
change of the deposit is div((1/2)(q/m) rho dt^2 grad phi); moving it to the
left-hand side gives div(eps0 (1 + chi) grad phi) with
chi = sum_s (q_s/m_s) rho_s dt^2 / (2 eps0).  A wrong factor in chi (beta = 1
instead of 1/2, a dropped eps0, q instead of q^2) breaks the identity at
first order, while the pusher alone fixes the true displacement.

The test loads a cold, neutral plasma on a lattice, displaces the electrons
by a small smooth field xi, and runs the oracle's deposit, solve, E and one
particle pass.  The final positions x^{n+1} are recovered from the stored
state by undoing the first push of the next step (cold particles: no
v_theta, no axis crossing, so x'' = x~ - v' dt exactly), redeposited, and
the residual  A_0 phi - f(rho(x^{n+1}))  (A_0 the finite-volume operator with
chi = 0, f the volume-integrated right-hand side, both of Sec. 2.5) is
compared with the susceptibility's own term T = (A_chi - A_0) phi.

Measured behaviour, which the assertions fix:
  - residual/T is a few 1e-3 to 1e-2; planted in the oracle, beta = 1 gives
    0.5, a dropped eps0 1e11, q/m in place of q^2/m (a dropped q) 1.0;
  - its part linear in the displacement (Richardson extrapolation in xi) is
    the discretisation mismatch between the particle deposit's response and
    the finite-volume operator, and falls 4x per mesh halving (second order);
  - the rest is quadratic in the displacement: the residual itself shrinks
    4x when xi halves.
Rows next to the z walls and the column next to r = R are left out: there
the gather uses the one-sided E of the Dirichlet nodes (first order, the
E = -grad phi reading of the boundary nodes), which the identity does not
survive at O(1).
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle

EPS0 = 8.8541878128e-12
N0 = 1e15
R, L = 0.05, 0.02


def _lattice(nz, nr, m):
    """m x m particles per cell, uniform in z and in r^2 (cell-centred)."""
    dz, dr = L / (nz - 1), R / (nr - 1)
    a = (np.arange(m) + 0.5) / m
    i, j, az, ar = np.meshgrid(np.arange(nz - 1), np.arange(nr - 1), a, a, indexing="ij")
    z = (i + az) * dz
    r = np.sqrt((j * dr) ** 2 + ar * (((j + 1) * dr) ** 2 - (j * dr) ** 2))
    w = N0 * np.pi * (((j + 1) * dr) ** 2 - (j * dr) ** 2) * dz / m ** 2
    return z.ravel(), r.ravel(), w.ravel()


def _cfg(nz, nr, wpdt, n):
    cfg = W.collisionless(W.config("c1"))
    cfg.update(nz=nz, nr=nr, R=R, L=L, mg_tol=1e-13, mg_max_cycles=300)
    cfg["rf"] = dict(amp=[0.0], freq=[W.F_RF], phase=[0.0])
    cfg["dt"] = wpdt / np.sqrt(N0 * W.QE ** 2 / (EPS0 * W.ME))
    cfg["species"] = [dict(sp, n0=N0, n_init=0, capacity=n + 16) for sp in cfg["species"]]
    return cfg


def residual_ratio(nz, nr, wpdt, delta, m=4):
    """max |A_0 phi - f(rho(x^{n+1}))| / max |T| over the interior nodes, for
    electrons displaced by xi = delta dz sin(pi z/L) cos(pi r/(2R))."""
    z0, r0, w = _lattice(nz, nr, m)
    n = len(z0)
    cfg = _cfg(nz, nr, wpdt, n)
    dz = L / (nz - 1)
    xi = delta * dz * np.sin(np.pi * z0 / L) * np.cos(np.pi * r0 / (2 * R))
    zero = np.zeros(n)
    o = Oracle(cfg, capacity=n + 16)
    cold = dict(r=r0, vr=zero, vt=zero, vz=zero, ar=zero, az=zero, w=w)
    o.set_particles(0, dict(cold, z=z0 + xi, id=np.arange(n, 2 * n, dtype=np.uint64)))
    o.set_particles(1, dict(cold, z=z0, id=np.arange(n, dtype=np.uint64)))
    o.deposit()
    o.finalize()
    chi = o.grid("chi")
    st, _, _ = o.solve(0.0)
    assert st == 0
    phi = o.grid("phi")
    o.efield()
    o.particle_pass()
    final = Oracle(cfg, capacity=n + 16)
    for s in (0, 1):
        p = o.get_particles(s)
        assert len(p["r"]) == n, "a particle reached a wall"
        assert np.all(p["vt"] == 0.0)
        p["z"] = p["z"] - p["vz"] * cfg["dt"]
        p["r"] = p["r"] - p["vr"] * cfg["dt"]
        final.set_particles(s, p)
    final.deposit()
    final.finalize()
    a0 = o.apply_A(np.zeros_like(chi), phi)
    t = o.apply_A(chi, phi) - a0
    res = a0 - o.rhs(final.grid("rho"))
    inner = (slice(2, nz - 2), slice(0, nr - 2))
    return float(np.abs(res[inner]).max() / np.abs(t[inner]).max())


MESHES = ((17, 33), (33, 65), (65, 129))


@pytest.mark.parametrize("wpdt", [0.5, 2.0, 5.0])
def test_final_charge_satisfies_poisson_to_second_order(wpdt):
    d = 0.02
    lin = []
    for nz, nr in MESHES:
        r1, r2, r4 = (residual_ratio(nz, nr, wpdt, d / k) for k in (1, 2, 4))
        # the identity holds to a few per cent of the chi term even on the
        # coarsest mesh; a wrong chi factor leaves 50-100 % of it
        assert max(r1, r2, r4) < 0.03, (nz, r1, r2, r4)
        # residual/T = A + B xi: A the discretisation part, B xi the
        # quadratic part of the residual.  A from the two smaller xi ...
        a = 2.0 * r4 - r2
        assert a > 0.0, (nz, r1, r2, r4)
        # ... predicts the largest one: the model holds
        assert abs((2.0 * r2 - r1) - a) < 0.1 * a, (nz, r1, r2, r4)
        # the nonlinear part halves with xi relative to T, i.e. the
        # residual's nonlinear part shrinks 4x when xi halves
        assert 1.7 < (r1 - a) / (r2 - a) < 2.3, (nz, r1, r2, r4)
        lin.append(a)
    # the discretisation part is second order in the mesh spacing
    for coarse, fine in zip(lin, lin[1:]):
        assert 3.3 < coarse / fine < 5.0, lin
