"""Collisionless window of the implicit r-z timestep, and the gradient of a
time-averaged ion-density functional, written out in plain PyTorch (FP64, CPU).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the CUDA path's
hand-written adjoint is checked against the gradient that PyTorch's autograd
takes through this forward.  It shares no code with the product library.

The forward is the oracle's timestep (``oracle.c``) with the Monte Carlo step
switched off (no collisions, no births, no splitting) and the field solve done
exactly (a dense solve of the interior finite-volume system) instead of by
multigrid; ``tests/test_oracle_window.py`` pins it to ``oracle.c``.  Steps, in
the paper's merged cycle (Sec. 2.1):

  rho, chi from the deposit (Eq. (10), Sec. 2.1) -> phi at t_{n+1}
  (Sec. 2.5, Eq. (11), Dirichlet electrodes: z = 0 at V(t), z = L at the
  given row, r = R at 0) -> E = -grad phi -> per particle: gather E at x~
  (Sec. 2.4), final push (Sec. 2.1, 2.3), axis reflection, walls, first push
  in the local X-Y frame with the rotation back (Sec. 2.3, Eqs. (4)-(5)),
  walls -> deposit at the new x~.

Functional: J = (1/K) sum over the K steps of sum over nodes w_k N_i(k),
N_i the ion deposit after each step's particle pass, i.e. the time average of
the integral of w n_i over the volume (n_i = N_i / V_k).  Parameters: the
amplitude of the first rf component and the potentials of the z = L row.

Conventions where the forward is not differentiable: a particle's cell is
piecewise constant (no gradient through the cell index); the axis reflection
takes |.| (derivative sign(.)); a particle that reaches a wall is frozen and
leaves the sums; the face susceptibility max(chi_lo, chi_hi) passes its
derivative to chi_lo when chi_lo > chi_hi and to chi_hi otherwise (ties to the
higher index, as the oracle's face rule picks it).
"""
from __future__ import annotations

import math

import numpy as np
import torch

EPS0 = 8.8541878128e-12


class Window:
    """The window's problem data (mesh, species, time step) from a workload dict."""

    def __init__(self, cfg: dict):
        self.cfg = cfg
        self.nz, self.nr = cfg["nz"], cfg["nr"]
        self.L, self.R = cfg["L"], cfg["R"]
        self.dz = self.L / (self.nz - 1)
        self.dr = self.R / (self.nr - 1)
        self.dt = cfg["dt"]
        self.q = [sp["q"] for sp in cfg["species"]]
        self.m = [sp["m"] for sp in cfg["species"]]
        self.zr2 = cfg.get("weighting", "zr2") == "zr2"
        self.mean_face = cfg.get("chi_face", "max") == "mean"
        rf = cfg["rf"]
        self.rf = [(float(a), float(f), float(p)) for a, f, p in zip(rf["amp"], rf["freq"], rf["phase"])]
        t = lambda a: torch.tensor(a, dtype=torch.float64)
        nz, nr, dz, dr = self.nz, self.nr, self.dz, self.dr
        j = np.arange(nr, dtype=np.float64)
        rp = (j + 0.5) * dr
        rm = np.where(j > 0, (j - 0.5) * dr, 0.0)
        self.area_z = t(math.pi * (rp * rp - rm * rm))          # z-face area of node j's control volume
        self.gz = self.area_z / dz                                # z-face geometry: area / dz
        self.gr = t(2.0 * math.pi * rp * dz / dr)                 # r-face (j, j+1) geometry
        self.V = t(self._node_volumes())

    def _node_volumes(self):
        """Node volumes of the deposit (Sec. 2.4; boundary rows and r = R take
        the inner part of the support)."""
        nz, nr, dz, dr = self.nz, self.nr, self.dz, self.dr
        r = np.arange(nr) * dr
        v = np.zeros(nr)
        for j in range(nr):
            if self.zr2:
                if j == 0:
                    v[j] = math.pi / 2 * r[1] ** 2
                elif j == nr - 1:
                    v[j] = math.pi / 2 * (r[j] ** 2 - r[j - 1] ** 2)
                else:
                    v[j] = math.pi / 2 * (r[j + 1] ** 2 - r[j - 1] ** 2)
            else:
                if j == 0:
                    v[j] = math.pi / 3 * r[1] ** 2
                elif j == nr - 1:
                    v[j] = math.pi / 3 * dr * (2 * r[j] + r[j - 1])
                else:
                    v[j] = math.pi / 3 * (r[j + 1] * (r[j] + r[j + 1]) - r[j - 1] * (r[j] + r[j - 1]))
        hz = np.full(nz, dz)
        hz[0] = hz[-1] = 0.5 * dz
        return hz[:, None] * v[None, :]

    # ---- particles <-> mesh (Sec. 2.4) ----
    def _cells(self, r, z):
        i = torch.clamp(torch.floor(z.detach() / self.dz), 0, self.nz - 2).long()
        j = torch.clamp(torch.floor(r.detach() / self.dr), 0, self.nr - 2).long()
        return i, j

    def _shape(self, r, z, i, j):
        z0 = i.double() * self.dz
        sz1 = (z - z0) / self.dz
        sz0 = 1.0 - sz1
        r0 = j.double() * self.dr
        r1 = r0 + self.dr
        if self.zr2:
            sr1 = (r * r - r0 * r0) / (r1 * r1 - r0 * r0)
        else:
            sr1 = (r - r0) / self.dr
        sr0 = 1.0 - sr1
        return (sz0, sz1), (sr0, sr1)

    def deposit(self, r, z, w):
        """N on the nodes: w times the shape factors (Eq. (9) or (8))."""
        i, j = self._cells(r, z)
        sz, sr = self._shape(r, z, i, j)
        N = torch.zeros(self.nz * self.nr, dtype=torch.float64)
        for a in (0, 1):
            for b in (0, 1):
                N = N.index_add(0, (i + a) * self.nr + (j + b), w * sz[a] * sr[b])
        return N.reshape(self.nz, self.nr)

    def gather(self, Ez, Er, r, z):
        i, j = self._cells(r, z)
        sz, sr = self._shape(r, z, i, j)
        ez = torch.zeros_like(r)
        er = torch.zeros_like(r)
        fz, fr = Ez.reshape(-1), Er.reshape(-1)
        for a in (0, 1):
            for b in (0, 1):
                k = (i + a) * self.nr + (j + b)
                ez = ez + sz[a] * sr[b] * fz[k]
                er = er + sz[a] * sr[b] * fr[k]
        return ez, er

    # ---- field (Sec. 2.5) ----
    def _face(self, lo, hi):
        if self.mean_face:
            return 0.5 * (lo + hi)
        return torch.where(lo > hi, lo, hi)

    def solve(self, rho, chi, V, phi_zL):
        """phi of the finite-volume system of Eq. (11) with the Dirichlet rows
        z = 0 (V, the corner at r = R grounded), z = L (phi_zL) and r = R (0);
        a dense solve of the interior unknowns."""
        nz, nr = self.nz, self.nr
        zero = torch.zeros((), dtype=torch.float64)
        row0 = torch.cat([V * torch.ones(nr - 1, dtype=torch.float64), zero.reshape(1)])
        interior_rows = torch.zeros(nz - 2, nr, dtype=torch.float64)
        phiB = torch.cat([row0.reshape(1, nr), interior_rows, phi_zL.reshape(1, nr)], 0)
        ni, nj = nz - 2, nr - 1                      # interior: i = 1..nz-2, j = 0..nr-2
        idx = -torch.ones(nz, nr, dtype=torch.long)
        idx[1:nz - 1, 0:nr - 1] = torch.arange(ni * nj).reshape(ni, nj)
        cz = (1.0 + self._face(chi[:-1, :], chi[1:, :])) * self.gz[None, :]       # face (i, i+1) at j
        cr = (1.0 + self._face(chi[:, :-1], chi[:, 1:])) * self.gr[None, :-1]     # face (j, j+1) at i
        n = ni * nj
        A = torch.zeros(n * n, dtype=torch.float64)
        rhs = (rho * self.area_z[None, :] * self.dz / EPS0)[1:nz - 1, 0:nr - 1].reshape(-1)
        I, Jc = torch.meshgrid(torch.arange(1, nz - 1), torch.arange(0, nr - 1), indexing="ij")
        I, Jc = I.reshape(-1), Jc.reshape(-1)
        p = idx[I, Jc]
        # the four faces of each interior node: (neighbour i, neighbour j, coefficient)
        faces = [(I - 1, Jc, cz[I - 1, Jc]), (I + 1, Jc, cz[I, Jc]),
                 (I, Jc + 1, cr[I, Jc])]
        jm = Jc > 0
        faces.append((I[jm], Jc[jm] - 1, cr[I[jm], Jc[jm] - 1]))
        for f, (qi, qj, c) in enumerate(faces):
            pp = p if f < 3 else p[jm]
            A = A.index_add(0, pp * n + pp, c)
            q = idx[qi, qj]
            inner = q >= 0
            A = A.index_add(0, pp[inner] * n + q[inner], -c[inner])
            rhs = rhs.index_add(0, pp[~inner], c[~inner] * phiB[qi[~inner], qj[~inner]])
        u = torch.linalg.solve(A.reshape(n, n), rhs)
        phi = phiB.clone()
        phi = phi.index_put((I, Jc), u)
        return phi

    def efield(self, phi):
        """E = -grad phi: central differences inside, one-sided on the z rows
        and at r = R, E_r = 0 on the axis."""
        dz, dr = self.dz, self.dr
        ez_in = -(phi[2:, :] - phi[:-2, :]) / (2 * dz)
        ez0 = -(phi[1:2, :] - phi[0:1, :]) / dz
        ezL = -(phi[-1:, :] - phi[-2:-1, :]) / dz
        Ez = torch.cat([ez0, ez_in, ezL], 0)
        er_in = -(phi[:, 2:] - phi[:, :-2]) / (2 * dr)
        er0 = torch.zeros_like(phi[:, 0:1])
        erR = -(phi[:, -1:] - phi[:, -2:-1]) / dr
        Er = torch.cat([er0, er_in, erR], 1)
        return Ez, Er

    def voltage(self, amp0, t):
        v = amp0 * math.sin(2 * math.pi * self.rf[0][1] * t + self.rf[0][2])
        for a, f, p in self.rf[1:]:
            v = v + a * math.sin(2 * math.pi * f * t + p)
        return v

    # ---- particles (Sec. 2.1, 2.3) ----
    def _inside(self, r, z):
        return (z > 0.0) & (z < self.L) & (r < self.R)

    def push(self, s, st, Ez, Er):
        """Final push at the gathered E, axis, walls, first push, walls.  A
        particle that reaches a wall keeps its state and leaves (alive False)."""
        r, z, vr, vt, vz, ar, az, alive = st
        dt, qm = self.dt, self.q[s] / self.m[s]
        ez, er = self.gather(Ez, Er, r, z)
        z1 = z + 0.5 * qm * ez * dt * dt
        rr = r + 0.5 * qm * er * dt * dt
        vz1 = vz + 0.5 * qm * ez * dt
        vr1 = vr + 0.5 * qm * er * dt
        az1 = 0.5 * (qm * ez + az)
        ar1 = 0.5 * (qm * er + ar)
        flip = (rr < 0.0).detach()
        r1 = torch.where(flip, -rr, rr)
        vr1 = torch.where(flip, torch.abs(vr1), vr1)
        ar1 = torch.where(flip, torch.abs(ar1), ar1)
        alive1 = alive & self._inside(r1.detach(), z1.detach())
        vx = vr1 + 0.5 * ar1 * dt
        vy = vt
        vz2 = vz1 + 0.5 * az1 * dt
        x = r1 + vx * dt
        y = vy * dt
        z2 = z1 + vz2 * dt
        q2 = x * x + y * y
        pos = (q2 > 0.0).detach()
        rn = torch.sqrt(torch.where(pos, q2, torch.ones_like(q2)))
        c = torch.where(pos, x / rn, torch.ones_like(x))
        sn = torch.where(pos, y / rn, torch.zeros_like(y))
        r2 = torch.where(pos, rn, torch.zeros_like(rn))
        vr2 = vx * c + vy * sn
        vt2 = -vx * sn + vy * c
        ar2 = ar1 * c
        alive2 = alive1 & self._inside(r2.detach(), z2.detach())
        keep = lambda new, old: torch.where(alive2, new, old)
        return (keep(r2, r), keep(z2, z), keep(vr2, vr), keep(vt2, vt), keep(vz2, vz), keep(ar2, ar),
                keep(az1, az), alive2)

    def run(self, parts, amp0, phi_zL, w_grid, K, step0=0, trace=None):
        """J over K steps from the particle states `parts` (per species a dict
        of r, z, vr, vt, vz, ar, az, w arrays) at step index step0.  amp0 and
        phi_zL may require grad.  `trace` (a list) receives per-step states."""
        T = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64))
        st = []
        ws = []
        for p in parts:
            st.append(tuple(T(p[k]) for k in ("r", "z", "vr", "vt", "vz", "ar", "az")) +
                      (torch.ones(len(p["r"]), dtype=torch.bool),))
            ws.append(T(p["w"]))
        w_grid = T(w_grid)
        N = [self.deposit(s_[0], s_[1], w * s_[7]) for s_, w in zip(st, ws)]
        J = torch.zeros((), dtype=torch.float64)
        for n in range(K):
            rho = sum(self.q[s] * N[s] / self.V for s in (0, 1))
            chi = sum(0.5 * (self.q[s] / self.m[s]) * self.q[s] * N[s] / self.V * self.dt * self.dt / EPS0
                      for s in (0, 1))
            t = (step0 + n + 1) * self.dt
            phi = self.solve(rho, chi, self.voltage(amp0, t), phi_zL)
            Ez, Er = self.efield(phi)
            st = [self.push(s, st[s], Ez, Er) for s in (0, 1)]
            N = [self.deposit(st[s][0], st[s][1], ws[s] * st[s][7]) for s in (0, 1)]
            J = J + (w_grid * N[1]).sum() / K
            if trace is not None:
                trace.append(dict(phi=phi.detach().clone(), st=[tuple(x.detach().clone() for x in s_) for s_ in st]))
        return J


def window_grad(cfg: dict, parts, w_grid, K, step0=0, amp0=None, phi_zL=None):
    """(J, dJ/d amp0, dJ/d phi_zL) by autograd through the window."""
    win = Window(cfg)
    a = torch.tensor(float(cfg["rf"]["amp"][0] if amp0 is None else amp0), dtype=torch.float64,
                     requires_grad=True)
    pz = np.zeros(cfg["nr"]) if phi_zL is None else np.asarray(phi_zL, dtype=np.float64)
    p = torch.tensor(pz, dtype=torch.float64, requires_grad=True)
    J = win.run(parts, a, p, w_grid, K, step0)
    J.backward()
    return float(J.detach()), float(a.grad), p.grad.numpy().copy()


def window_J(cfg: dict, parts, w_grid, K, step0=0, amp0=None, phi_zL=None, trace=None):
    """J alone (finite-difference checks)."""
    win = Window(cfg)
    with torch.no_grad():
        a = torch.tensor(float(cfg["rf"]["amp"][0] if amp0 is None else amp0), dtype=torch.float64)
        pz = np.zeros(cfg["nr"]) if phi_zL is None else np.asarray(phi_zL, dtype=np.float64)
        return float(win.run(parts, a, torch.tensor(pz, dtype=torch.float64), w_grid, K, step0, trace))
