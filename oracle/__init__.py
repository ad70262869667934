"""Plain FP64 CPU oracle of the implicit r-z PIC/MC timestep (arXiv:1001.2969).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the product library (``paper_1001_2969_gb300``) and does not import it.

The arithmetic lives in ``oracle.c`` (C99, FP64, serial, built with
``-ffp-contract=off``); this module only marshals arguments with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

ELASTIC, EXCITE, IONIZE, CX = 0, 1, 2, 3
KIND = {"elastic": ELASTIC, "excite": EXCITE, "ionize": IONIZE, "cx": CX}
GRID = {"Ne": 0, "Ni": 1, "rho": 2, "chi": 3, "phi": 4, "Ez": 5, "Er": 6}

# counter layout (mirrors oracle.h)
C_COLL, C_CAND, C_NUOVER, C_BIRTHS, C_SPLITS, C_ABS, C_NCOUNT = 0, 8, 10, 12, 14, 16, 24


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain IEEE FP64, no FMA contraction)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)


class OrcConfig(C.Structure):
    _fields_ = [
        ("R", C.c_double), ("L", C.c_double), ("nz", C.c_int32), ("nr", C.c_int32),
        ("q", C.c_double * 2), ("m", C.c_double * 2), ("n0", C.c_double * 2),
        ("T_eV", C.c_double * 2), ("n_init", C.c_int64 * 2),
        ("xs_ne", C.c_int32 * 2), ("xs_emax", C.c_double * 2), ("xs_nch", C.c_int32 * 2),
        ("xs_sigma", _dp * 2), ("xs_thr", _dp * 2), ("xs_kind", _ip * 2), ("xs_B", C.c_double * 2),
        ("rf_n", C.c_int32), ("rf_amp", _dp), ("rf_freq", _dp), ("rf_phase", _dp),
        ("p_Pa", C.c_double), ("T_K", C.c_double), ("m_gas", C.c_double),
        ("dt", C.c_double), ("seed", C.c_uint64),
        ("weighting", C.c_int32), ("chi_face", C.c_int32), ("scatter", C.c_int32),
        ("split_every", C.c_int32), ("mg_max_cycles", C.c_int32), ("mg_tol", C.c_double),
        ("phi_zL", _dp), ("eedf_bins", C.c_int32), ("eedf_emax", C.c_double),
        ("circuit_C", C.c_double),
        ("pusher", C.c_int32),
        ("ion_subcycle", C.c_int32),
        ("mg_guess", C.c_int32),
    ]


def _declare(L):
    vp = C.c_void_p
    L.orc_create.restype = vp
    L.orc_create.argtypes = [C.POINTER(OrcConfig), C.c_int64]
    L.orc_destroy.argtypes = [vp]
    L.orc_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.orc_count.restype = C.c_int64
    L.orc_count.argtypes = [vp, C.c_int]
    L.orc_set_particles.argtypes = [vp, C.c_int, C.c_int64] + [_dp] * 8 + [_u64p]
    L.orc_get_particles.argtypes = [vp, C.c_int] + [_dp] * 8 + [_u64p]
    L.orc_set_next_id.argtypes = [vp, C.c_int, C.c_uint64]
    L.orc_get_next_id.restype = C.c_uint64
    L.orc_get_next_id.argtypes = [vp, C.c_int]
    L.orc_set_step.argtypes = [vp, C.c_int64]
    L.orc_get_step.restype = C.c_int64
    L.orc_get_step.argtypes = [vp]
    L.orc_ion_pass.restype = C.c_int
    L.orc_ion_pass.argtypes = [vp]
    L.orc_merge.restype = C.c_int64
    L.orc_merge.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double)]
    L.orc_load.argtypes = [vp]
    L.orc_load_range.argtypes = [vp, C.c_int, C.c_int64, C.c_int64] + [_dp] * 8 + [_u64p]
    L.orc_deposit.argtypes = [vp]
    L.orc_finalize.argtypes = [vp]
    L.orc_node_volumes.argtypes = [vp, _dp]
    L.orc_get_grid.argtypes = [vp, C.c_int, _dp]
    L.orc_set_grid.argtypes = [vp, C.c_int, _dp]
    L.orc_voltage.restype = C.c_double
    L.orc_voltage.argtypes = [vp, C.c_double]
    L.orc_solve.restype = C.c_int
    L.orc_solve.argtypes = [vp, C.c_double, C.c_double, C.c_int, _ip, _dp]
    L.orc_apply_A.argtypes = [vp, _dp, _dp, _dp]
    L.orc_rhs.argtypes = [vp, _dp, _dp]
    L.orc_efield.argtypes = [vp]
    L.orc_particle_pass.argtypes = [vp]
    L.orc_step.argtypes = [vp, C.c_int, _ip, _dp]
    L.orc_get_counters.argtypes = [vp, _i64p, _dp]
    L.orc_reset_counters.argtypes = [vp]
    L.orc_get_moments.argtypes = [vp] + [_dp] * 6 + [_i64p]
    L.orc_reset_moments.argtypes = [vp]
    L.orc_sigma.restype = C.c_double
    L.orc_sigma.argtypes = [vp, C.c_int, C.c_int, C.c_double]
    L.orc_nu_max.restype = C.c_double
    L.orc_nu_max.argtypes = [vp, C.c_int]
    L.orc_p_null.restype = C.c_double
    L.orc_p_null.argtypes = [vp, C.c_int]
    L.orc_cos_chi.restype = C.c_double
    L.orc_cos_chi.argtypes = [vp, C.c_double, C.c_double]
    L.orc_scatter_dir.argtypes = [C.c_double] * 5 + [_dp]
    L.orc_ejected_energy.restype = C.c_double
    L.orc_ejected_energy.argtypes = [C.c_double] * 4
    L.orc_get_circuit.argtypes = [vp, _dp]
    L.orc_get_at.argtypes = [vp, C.c_int, _dp]
    L.orc_set_at.argtypes = [vp, C.c_int, _dp]
    L.orc_w_ref.restype = C.c_double
    L.orc_w_ref.argtypes = [vp, C.c_int, C.c_int]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def philox(ctr, key):
    """Philox4x32-10 block: four 32-bit counter words, two key words."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return [int(x) for x in o]


FIELDS = ("r", "z", "vr", "vt", "vz", "ar", "az", "w")


class Oracle:
    """One oracle instance (a simulation state) built from a workload dict."""

    def __init__(self, cfg: dict, capacity: int | None = None):
        self.cfg = cfg
        L = lib()
        self._keep = []
        c = OrcConfig()
        c.R, c.L, c.nz, c.nr = cfg["R"], cfg["L"], cfg["nz"], cfg["nr"]
        for s, sp in enumerate(cfg["species"]):
            c.q[s], c.m[s], c.n0[s], c.T_eV[s] = sp["q"], sp["m"], sp["n0"], sp["T_eV"]
            c.n_init[s] = sp["n_init"]
            xs = cfg["xsec"][s]
            sig = _d(xs["sigma"]).reshape(-1)
            thr = _d(xs["threshold"])
            kind = np.ascontiguousarray([KIND[k] if isinstance(k, str) else k for k in xs["kind"]],
                                        dtype=np.int32)
            self._keep += [sig, thr, kind]
            c.xs_ne[s] = xs["n_e"]
            c.xs_emax[s] = xs["E_max"]
            c.xs_nch[s] = len(kind)
            c.xs_sigma[s] = _ptr(sig)
            c.xs_thr[s] = _ptr(thr)
            c.xs_kind[s] = _ptr(kind, _ip)
            c.xs_B[s] = xs.get("B_eV", 10.0)
        amp, freq, ph = (_d(cfg["rf"][k]) for k in ("amp", "freq", "phase"))
        self._keep += [amp, freq, ph]
        c.rf_n = len(amp)
        c.rf_amp, c.rf_freq, c.rf_phase = _ptr(amp), _ptr(freq), _ptr(ph)
        g = cfg["gas"]
        c.p_Pa, c.T_K, c.m_gas = g["p_Pa"], g["T_K"], g["m_gas"]
        c.dt = cfg["dt"]
        c.seed = cfg["seed"]
        c.weighting = {"zr2": 0, "zr": 1}[cfg.get("weighting", "zr2")]
        c.chi_face = {"max": 0, "mean": 1}[cfg.get("chi_face", "max")]
        c.scatter = {"vs": 0, "isotropic": 1}[cfg.get("scatter", "vs")]
        c.split_every = cfg.get("split_every", 0)
        c.mg_max_cycles = cfg.get("mg_max_cycles", 50)
        c.mg_tol = cfg.get("mg_tol", 1e-10)
        if cfg.get("phi_zL") is not None:
            pz = _d(cfg["phi_zL"])
            self._keep.append(pz)
            c.phi_zL = _ptr(pz)
        c.eedf_bins = cfg.get("eedf_bins", 0)
        c.eedf_emax = cfg.get("eedf_emax", 100.0)
        c.circuit_C = float(cfg.get("circuit_C", 0.0))
        c.pusher = {"local": 0, "xyz": 1}[cfg.get("pusher", "local")]
        c.ion_subcycle = int(cfg.get("ion_subcycle", 1))
        c.mg_guess = {"previous": 0, "linear": 1}[cfg.get("mg_guess", "linear")]
        if capacity is None:
            capacity = max(int(1.5 * max(sp["capacity"] for sp in cfg["species"])), 64)
        self.capacity = capacity
        self._c = c
        self.h = L.orc_create(C.byref(c), capacity)
        self.nz, self.nr = cfg["nz"], cfg["nr"]

    def __del__(self):
        try:
            if self.h:
                lib().orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # particles
    def count(self, s):
        return lib().orc_count(self.h, s)

    def load(self):
        lib().orc_load(self.h)

    def load_range(self, s, p0, p1):
        n = p1 - p0
        arr = {k: np.zeros(n) for k in FIELDS}
        idv = np.zeros(n, dtype=np.uint64)
        lib().orc_load_range(self.h, s, p0, p1, *[_ptr(arr[k]) for k in FIELDS], _ptr(idv, _u64p))
        arr["id"] = idv
        return arr

    def set_particles(self, s, p: dict):
        n = len(p["r"])
        arrs = [_d(p[k]) for k in FIELDS]
        idv = np.ascontiguousarray(p["id"], dtype=np.uint64)
        lib().orc_set_particles(self.h, s, n, *[_ptr(a) for a in arrs], _ptr(idv, _u64p))

    def get_particles(self, s) -> dict:
        n = self.count(s)
        arr = {k: np.zeros(n) for k in FIELDS}
        idv = np.zeros(n, dtype=np.uint64)
        lib().orc_get_particles(self.h, s, *[_ptr(arr[k]) for k in FIELDS], _ptr(idv, _u64p))
        arr["id"] = idv
        return arr

    def get_at(self, s) -> np.ndarray:
        """a_theta of species s (the X-Y-Z pusher carries it)."""
        out = np.zeros(self.count(s))
        lib().orc_get_at(self.h, s, _ptr(out))
        return out

    def set_at(self, s, at):
        a = _d(at)
        assert len(a) == self.count(s)
        lib().orc_set_at(self.h, s, _ptr(a))

    def set_next_id(self, s, v):
        lib().orc_set_next_id(self.h, s, int(v))

    def next_id(self, s):
        return lib().orc_get_next_id(self.h, s)

    def set_step(self, n):
        lib().orc_set_step(self.h, int(n))

    def step_index(self):
        return lib().orc_get_step(self.h)

    def merge(self, s, frac, dv):
        """Merge light particles of species s in pairs; (pairs, energy lost in J)."""
        e = C.c_double(0)
        n = lib().orc_merge(self.h, s, float(frac), float(dv), C.byref(e))
        return int(n), e.value

    def ion_pass(self):
        """True when the next pass moves the ions (ion subcycling)."""
        return bool(lib().orc_ion_pass(self.h))

    # grids
    def deposit(self):
        lib().orc_deposit(self.h)

    def finalize(self):
        lib().orc_finalize(self.h)

    def grid(self, name) -> np.ndarray:
        out = np.zeros((self.nz, self.nr))
        lib().orc_get_grid(self.h, GRID[name], _ptr(out))
        return out

    def set_grid(self, name, a):
        a = _d(a)
        lib().orc_set_grid(self.h, GRID[name], _ptr(a))

    def node_volumes(self):
        out = np.zeros((self.nz, self.nr))
        lib().orc_node_volumes(self.h, _ptr(out))
        return out

    def voltage(self, t):
        return lib().orc_voltage(self.h, t)

    def solve(self, V, tol=None, max_cycles=None):
        tol = self.cfg.get("mg_tol", 1e-10) if tol is None else tol
        max_cycles = self.cfg.get("mg_max_cycles", 50) if max_cycles is None else max_cycles
        cyc = C.c_int32(0)
        res = C.c_double(0)
        st = lib().orc_solve(self.h, V, tol, max_cycles, C.byref(cyc), C.byref(res))
        return st, cyc.value, res.value

    def apply_A(self, chi, u):
        chi, u = _d(chi), _d(u)
        out = np.zeros((self.nz, self.nr))
        lib().orc_apply_A(self.h, _ptr(chi), _ptr(u), _ptr(out))
        return out

    def rhs(self, rho):
        rho = _d(rho)
        out = np.zeros((self.nz, self.nr))
        lib().orc_rhs(self.h, _ptr(rho), _ptr(out))
        return out

    def efield(self):
        lib().orc_efield(self.h)

    def particle_pass(self):
        lib().orc_particle_pass(self.h)

    def step(self, n=1):
        cyc = C.c_int32(0)
        res = C.c_double(0)
        lib().orc_step(self.h, n, C.byref(cyc), C.byref(res))
        return cyc.value, res.value

    def counters(self):
        c = np.zeros(C_NCOUNT, dtype=np.int64)
        q = np.zeros(3)
        lib().orc_get_counters(self.h, _ptr(c, _i64p), _ptr(q))
        return c, q

    def reset_counters(self):
        lib().orc_reset_counters(self.h)

    def moments(self):
        g = {k: np.zeros((self.nz, self.nr)) for k in ("ne", "ni", "phi", "Ez", "Er")}
        nb = max(self.cfg.get("eedf_bins", 0), 1)
        eedf = np.zeros(nb)
        n = C.c_int64(0)
        lib().orc_get_moments(self.h, *[_ptr(g[k]) for k in ("ne", "ni", "phi", "Ez", "Er")],
                              _ptr(eedf), C.byref(n))
        g["eedf"] = eedf[: self.cfg.get("eedf_bins", 0)]
        g["nsamples"] = n.value
        return g

    def reset_moments(self):
        lib().orc_reset_moments(self.h)

    # pieces
    def sigma(self, s, ch, E):
        return lib().orc_sigma(self.h, s, ch, E)

    def nu_max(self, s):
        return lib().orc_nu_max(self.h, s)

    def p_null(self, s):
        return lib().orc_p_null(self.h, s)

    def cos_chi(self, eps, R):
        return lib().orc_cos_chi(self.h, eps, R)

    def circuit(self):
        """(electrode voltage V, electrode charge Q, capacitor charge Q_c) after the last step."""
        out = np.zeros(3)
        lib().orc_get_circuit(self.h, _ptr(out))
        return tuple(out)

    def w_ref(self, s, j):
        return lib().orc_w_ref(self.h, s, j)


def scatter_dir(ux, uy, uz, cos_chi, phi):
    out = (C.c_double * 3)()
    lib().orc_scatter_dir(ux, uy, uz, cos_chi, phi, out)
    return np.array(list(out))


def ejected_energy(eps, thr, B, R):
    return lib().orc_ejected_energy(eps, thr, B, R)
