"""Seeded synthetic workloads for the r-z PIC/MC timestep (arXiv:1001.2969).

This module is the one place both the product path and the oracle take their
inputs from.  It holds no arithmetic of the method: only problem parameters
(the reactor geometry, gas, species, rf waveform and time step of the paper's
Sec. 3 benchmark and of the synthetic stand-ins for it), tabulated synthetic
cross sections, and random particle states for the parity tests.

The paper's own cross-section data (Phelps, argon) is not available, so the
tables are synthetic analytic forms sampled on a uniform grid: electron
elastic 1e-19 m^2, excitation from 11.5 eV and ionisation from 15.76 eV each
rising linearly to a peak and falling as 1/E beyond it, ion charge exchange
5e-19 m^2.
"""
from __future__ import annotations

import numpy as np

# CODATA 2018 / IUPAC values (problem parameters)
QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
M_AR = 39.948 * AMU
KB = 1.380649e-23

F_RF = 13.56e6


def _linear_rise_then_inv(E, thr, e_peak, s_peak):
    """sigma = s_peak (E - thr)/(e_peak - thr) on (thr, e_peak], s_peak e_peak / E above."""
    E = np.asarray(E, dtype=np.float64)
    out = np.zeros_like(E)
    rise = (E > thr) & (E <= e_peak)
    out[rise] = s_peak * (E[rise] - thr) / (e_peak - thr)
    hi = E > e_peak
    out[hi] = s_peak * e_peak / E[hi]
    return out


def argon_tables(E_max: float, n_e: int = 1001, with_inelastic: bool = True):
    """Synthetic argon cross sections on the uniform grid [0, E_max] (eV)."""
    E = np.linspace(0.0, E_max, n_e)
    el = np.full_like(E, 1e-19)
    sig = [el]
    thr = [0.0]
    kind = ["elastic"]
    if with_inelastic:
        sig.append(_linear_rise_then_inv(E, 11.5, 25.0, 2e-20))
        thr.append(11.5)
        kind.append("excite")
        sig.append(_linear_rise_then_inv(E, 15.76, 100.0, 3e-20))
        thr.append(15.76)
        kind.append("ionize")
    e_xs = dict(n_e=n_e, E_max=float(E_max), sigma=np.stack(sig), threshold=np.array(thr),
                kind=kind, B_eV=10.0)
    i_xs = dict(n_e=n_e, E_max=float(E_max), sigma=np.full((1, n_e), 5e-19),
                threshold=np.array([0.0]), kind=["cx"], B_eV=10.0)
    return [e_xs, i_xs]


def _species(n0, n, Te=3.0, Ti=0.026, cap_factor=1.5):
    cap = int(n * cap_factor) + 4096
    return [dict(q=-QE, m=ME, n0=n0, T_eV=Te, n_init=n, capacity=cap),
            dict(q=QE, m=M_AR, n0=n0, T_eV=Ti, n_init=n, capacity=cap)]


def config(name: str, **over) -> dict:
    """Workload by name.

    c1  small axisymmetric argon CCP: R 5 cm, gap 2 cm, 33 x 65 nodes,
        1e5 + 1e5 particles, n0 1e15 m^-3, 4 Pa, 100 V at 13.56 MHz,
        dt = T_rf/400, 200 steps.
    c2  production-size reactor (R >> L): R 20 cm, gap 2.5 cm, 129 x 513,
        1e7 + 1e7 particles, n0 5e15, 4 Pa, 300 V at 13.56 MHz,
        dt = T_rf/200, 2000 steps.
    c3  large dual-frequency reactor: R 30 cm, gap 3 cm, 257 x 1025,
        1e8 + 1e8 particles, n0 5e15, 8 Pa, 200 V at 60 MHz + 500 V at 2 MHz,
        dt = T_60MHz/100, 1000 steps.
    tiny  a few particles on a 5 x 5 mesh (brute-force cross-checks).
    """
    if name == "c1":
        amp = [100.0]
        cfg = dict(R=0.05, L=0.02, nz=33, nr=65, species=_species(1e15, 100_000),
                   rf=dict(amp=amp, freq=[F_RF], phase=[0.0]),
                   gas=dict(p_Pa=4.0, T_K=300.0, m_gas=M_AR),
                   dt=1.0 / F_RF / 400, steps=200, split_every=400)
    elif name == "c2":
        amp = [300.0]
        # room for the periodic split (every 200 steps), which multiplies the
        # particles that drifted to smaller radii
        cfg = dict(R=0.20, L=0.025, nz=129, nr=513, species=_species(5e15, 10_000_000, cap_factor=3.0),
                   rf=dict(amp=amp, freq=[F_RF], phase=[0.0]),
                   gas=dict(p_Pa=4.0, T_K=300.0, m_gas=M_AR),
                   dt=1.0 / F_RF / 200, steps=2000, split_every=200)
    elif name == "c3":
        amp = [200.0, 500.0]
        cfg = dict(R=0.30, L=0.03, nz=257, nr=1025, species=_species(5e15, 100_000_000, cap_factor=3.0),
                   rf=dict(amp=amp, freq=[60e6, 2e6], phase=[0.0, 0.0]),
                   gas=dict(p_Pa=8.0, T_K=300.0, m_gas=M_AR),
                   dt=1.0 / 60e6 / 100, steps=1000, split_every=100)
    elif name == "c5":
        # the adjoint window: collisionless (the cross sections are zero,
        # see collisionless()), 256 steps, checkpoints every 16
        amp = [100.0]
        cfg = dict(R=0.10, L=0.02, nz=65, nr=257, species=_species(1e15, 1_000_000),
                   rf=dict(amp=amp, freq=[F_RF], phase=[0.0]),
                   gas=dict(p_Pa=4.0, T_K=300.0, m_gas=M_AR),
                   dt=1.0 / F_RF / 200, steps=256, split_every=0, ckpt=16,
                   w_centre=(0.03, 0.01), w_sigma=0.005)
    elif name == "tiny":
        amp = [50.0]
        cfg = dict(R=0.004, L=0.004, nz=5, nr=5, species=_species(1e15, 8, cap_factor=64),
                   rf=dict(amp=amp, freq=[F_RF], phase=[0.0]),
                   gas=dict(p_Pa=4.0, T_K=300.0, m_gas=M_AR),
                   dt=1.0 / F_RF / 400, steps=4, split_every=0)
    else:
        raise KeyError(name)
    # table range: four times the summed electrode amplitude, in eV
    cfg["xsec"] = argon_tables(4.0 * sum(abs(a) for a in amp))
    if name == "c5":
        cfg["xsec"] = collisionless(cfg)["xsec"]
    cfg.update(dict(seed=1, weighting="zr2", chi_face="max", scatter="vs", mg_max_cycles=50,
                    mg_tol=1e-10, phi_zL=None, eedf_bins=200, eedf_emax=100.0,
                    precision="fp64"))
    cfg["name"] = name
    for k, v in over.items():
        cfg[k] = v
    return cfg


def batch_configs(n: int = 64, seed: int = 4, n_lo: int = 50_000, n_hi: int = 5_000_000,
                  precision: str = "mixed") -> list:
    """The batched sweep (c4): n independent argon reactors drawn from `seed`.

    Mesh nz in {33, 65, 129} and nr in {65, ..., 513} (at least 2 nz - 1)
    with c2's cell size (R and L follow the mesh), particles per species
    log-uniform in [n_lo, n_hi], pressure log-uniform in [1, 100] Pa, voltage
    uniform in [50, 500] V at 13.56 MHz, n0 5e15 m^-3, dt = T_rf/200; reactor k
    takes Philox seed 1000 + k.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nz = int(rng.choice([33, 65, 129]))
        nr_opts = [r for r in (65, 129, 257, 513) if r >= 2 * nz - 1]
        nr = int(rng.choice(nr_opts))
        npart = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        p = float(np.exp(rng.uniform(np.log(1.0), np.log(100.0))))
        v = float(rng.uniform(50.0, 500.0))
        cfg = dict(R=0.20 * (nr - 1) / 512, L=0.025 * (nz - 1) / 128, nz=nz, nr=nr,
                   species=_species(5e15, npart),
                   rf=dict(amp=[v], freq=[F_RF], phase=[0.0]),
                   gas=dict(p_Pa=p, T_K=300.0, m_gas=M_AR),
                   dt=1.0 / F_RF / 200, steps=500, split_every=200)
        cfg["xsec"] = argon_tables(4.0 * v)
        cfg.update(dict(seed=1000 + k, weighting="zr2", chi_face="max", scatter="vs",
                        mg_max_cycles=50, mg_tol=1e-10, phi_zL=None, eedf_bins=200,
                        eedf_emax=100.0, precision=precision))
        cfg["name"] = f"c4-{k}"
        out.append(cfg)
    return out


def collisionless(cfg: dict) -> dict:
    """Same workload with every cross section zero: no null-collision
    candidates, hence no collisions and no births (the adjoint window)."""
    out = dict(cfg)
    xs = []
    for t in cfg["xsec"]:
        t = dict(t)
        t["sigma"] = np.zeros_like(np.asarray(t["sigma"], dtype=np.float64))
        xs.append(t)
    out["xsec"] = xs
    out["split_every"] = 0
    return out


def gaussian_weight(cfg: dict, centre=None, sigma=None) -> np.ndarray:
    """Nodal weight w(r, z) of the adjoint window's functional: a Gaussian of
    width sigma (m) centred at (r, z) = centre (m), on the (nz, nr) nodes."""
    centre = cfg.get("w_centre", (0.03, 0.01)) if centre is None else centre
    sigma = cfg.get("w_sigma", 0.005) if sigma is None else sigma
    z = np.linspace(0.0, cfg["L"], cfg["nz"])[:, None]
    r = np.linspace(0.0, cfg["R"], cfg["nr"])[None, :]
    return np.exp(-((r - centre[0]) ** 2 + (z - centre[1]) ** 2) / (2.0 * sigma ** 2))


def scaled(cfg: dict, n_per_species: int) -> dict:
    """Same workload with a different particle count (capacity follows, in the
    same proportion)."""
    out = dict(cfg)
    out["species"] = [dict(sp) for sp in cfg["species"]]
    for sp in out["species"]:
        ratio = (sp["capacity"] - 4096) / sp["n_init"] if sp.get("n_init") else 1.5
        sp["n_init"] = int(n_per_species)
        sp["capacity"] = int(n_per_species * ratio) + 4096
    return out


def random_particles(cfg: dict, s: int, n: int, seed: int, hot: float = 1.0,
                     accel: float = 0.0, wscale: float = 1.0, margin: float = 0.0,
                     id0: int = 0) -> dict:
    """Random particle state of species s inside the domain (parity inputs).

    Positions are uniform in (z, r^2) in [margin, L - margin] x [0, R - margin],
    velocities normal with standard deviation hot * sqrt(T/m), accelerations
    normal with standard deviation `accel` (m/s^2), weights log-uniform over a
    decade around `wscale`, ids a random permutation of id0 .. id0+n-1.
    """
    rng = np.random.default_rng(seed)
    sp = cfg["species"][s]
    L, R = cfg["L"], cfg["R"]
    z = rng.uniform(margin, L - margin, n)
    r = np.sqrt(rng.uniform(0.0, (R - margin) ** 2, n))
    sig = hot * np.sqrt(sp["T_eV"] * QE / sp["m"])
    v = rng.normal(0.0, sig, (3, n))
    a = rng.normal(0.0, accel, (2, n)) if accel > 0 else np.zeros((2, n))
    w = wscale * 10.0 ** rng.uniform(-0.5, 0.5, n)
    ids = (rng.permutation(n) + id0).astype(np.uint64)
    return dict(r=r, z=z, vr=v[0], vt=v[1], vz=v[2], ar=a[0], az=a[1], w=w, id=ids)


def random_grid(cfg: dict, seed: int, scale: float = 1.0, smooth: bool = True) -> np.ndarray:
    """Random non-negative nodal field on the mesh (susceptibility / density inputs)."""
    rng = np.random.default_rng(seed)
    nz, nr = cfg["nz"], cfg["nr"]
    if smooth:
        zz = np.linspace(0, 1, nz)[:, None]
        rr = np.linspace(0, 1, nr)[None, :]
        k = rng.uniform(0.5, 2.5, 4)
        ph = rng.uniform(0, 2 * np.pi, 4)
        f = (1.0 + 0.5 * np.sin(np.pi * k[0] * zz + ph[0]) * np.cos(np.pi * k[1] * rr + ph[1])
             + 0.3 * np.sin(np.pi * k[2] * zz * rr + ph[2]))
        return scale * np.clip(f, 0.05, None)
    return scale * rng.uniform(0.0, 1.0, (nz, nr))
