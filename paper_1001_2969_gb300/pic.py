"""Thin ctypes binding of libpic.so (include/pic.h), the GB300 implicit
electrostatic PIC/MC timestep in axisymmetric r-z geometry (arXiv:1001.2969).

The functions keep the C names and only marshal arguments: every step of the
method runs in the library's CUDA kernels.  PyTorch supplies device memory
(its caching allocator, through the library's allocation hooks) and the
current CUDA stream.  Importing this module fails loudly when the library
has not been built; creating a handle fails loudly without a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK, PIC_ERR_ARG, PIC_ERR_CAPACITY, PIC_ERR_CUDA = 0, 1, 2, 3
PIC_ERR_NOT_CONVERGED, PIC_ERR_NUMERIC, PIC_ERR_TIMEOUT, PIC_ERR_STATE = 4, 5, 6, 7
PIC_FP64, PIC_MIXED = 0, 1
PIC_C_COLL, PIC_C_CAND, PIC_C_NUOVER, PIC_C_BIRTHS = 0, 8, 10, 12
PIC_C_SPLITS, PIC_C_ABS, PIC_C_MGCYC, PIC_C_STEPS, PIC_C_PSTEPS, PIC_NCOUNT = 14, 16, 22, 23, 24, 25
PIC_MAX_CH = 4
N_TIMING = 5
KIND = {"elastic": 0, "excite": 1, "ionize": 2, "cx": 3}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class pic_mesh(C.Structure):
    _fields_ = [("R", C.c_double), ("L", C.c_double), ("nz", C.c_int32), ("nr", C.c_int32)]


class pic_species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n0", C.c_double), ("T_eV", C.c_double),
                ("n_init", C.c_int64), ("capacity", C.c_int64)]


class pic_xsec(C.Structure):
    _fields_ = [("n_e", C.c_int32), ("E_max_eV", C.c_double), ("n_ch", C.c_int32),
                ("sigma_m2", _dp), ("threshold_eV", _dp), ("kind", _ip), ("B_eV", C.c_double)]


class pic_rf(C.Structure):
    _fields_ = [("n", C.c_int32), ("amp_V", _dp), ("freq_Hz", _dp), ("phase_rad", _dp)]


class pic_gas(C.Structure):
    _fields_ = [("p_Pa", C.c_double), ("T_K", C.c_double), ("m_gas", C.c_double)]


class pic_config(C.Structure):
    _fields_ = [("mesh", pic_mesh), ("sp", pic_species * 2), ("xs", pic_xsec * 2), ("rf", pic_rf),
                ("gas", pic_gas), ("dt", C.c_double), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("weighting", C.c_int32), ("chi_face", C.c_int32),
                ("scatter", C.c_int32), ("split_every", C.c_int32), ("mg_max_cycles", C.c_int32),
                ("mg_tol", C.c_double), ("phi_zL", _dp), ("births_capacity", C.c_int64),
                ("eedf_bins", C.c_int32), ("eedf_emax_eV", C.c_double), ("load", C.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("stream", C.c_void_p), ("circuit_C", C.c_double), ("pusher", C.c_int32),
                ("ion_subcycle", C.c_int32), ("mg_guess", C.c_int32)]


class pic_particles_view(C.Structure):
    _fields_ = [("n", C.c_int64), ("r", _dp), ("z", _dp), ("vr", _dp), ("vt", _dp), ("vz", _dp),
                ("ar", _dp), ("az", _dp), ("w", _dp), ("id", _u64p), ("cell", _ip), ("at", _dp)]


class pic_solve_info(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("rel_residual", C.c_double)]


class pic_moments_out(C.Structure):
    _fields_ = [("ne", _dp), ("ni", _dp), ("phi", _dp), ("Er", _dp), ("Ez", _dp), ("eedf", _dp),
                ("counters", _i64p), ("charge", _dp), ("nsamples", C.c_int64),
                ("on_device", C.c_int32)]


SYMBOLS = ("pic_init", "pic_step", "pic_field_solve", "pic_moments", "pic_get_particles",
           "pic_set_particles", "pic_set_step", "pic_set_boundary", "pic_get_fields",
           "pic_get_counts", "pic_save", "pic_load", "pic_profile", "pic_timings", "pic_destroy",
           "pic_last_error", "pic_status_string", "pic_field_solve_noalloc", "pic_batch_init",
           "pic_batch_step", "pic_batch_destroy", "pic_tune", "pic_get_circuit", "pic_window",
           "pic_merge", "pic_selftest_wait", "pic_fp64_fma_rate", "pic_get_deposit",
           "pic_set_deposit", "pic_set_id_stride")


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def lib():
    """The loaded library; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpic.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.pic_init.argtypes = [C.POINTER(pic_config), C.POINTER(vp)]
        L.pic_step.argtypes = [vp, C.c_int32]
        L.pic_batch_init.argtypes = [C.POINTER(vp), C.c_int32, vp, C.POINTER(vp)]
        L.pic_batch_step.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
        L.pic_batch_destroy.argtypes = [vp]
        L.pic_batch_destroy.restype = None
        L.pic_tune.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
        L.pic_get_circuit.argtypes = [vp, _dp]
        L.pic_merge.argtypes = [vp, C.c_int32, C.c_double, C.c_double, _i64p, _dp]
        L.pic_selftest_wait.argtypes = [C.c_int64, C.POINTER(C.c_int32)]
        L.pic_fp64_fma_rate.argtypes = [C.c_int32, _dp]
        L.pic_get_deposit.argtypes = [vp, vp, vp, vp, C.c_int32]
        L.pic_set_deposit.argtypes = [vp, vp, vp, vp, C.c_int32]
        L.pic_set_id_stride.argtypes = [vp, _u64p, C.c_uint64]
        L.pic_window.argtypes = [vp, C.c_int32, C.c_int32, _dp, C.c_double, _dp, C.c_int32, _dp, _dp, _dp]
        L.pic_field_solve.argtypes = [vp, vp, vp, C.c_double, vp, C.c_int32,
                                      C.POINTER(pic_solve_info)]
        L.pic_moments.argtypes = [vp, C.POINTER(pic_moments_out), C.c_int32]
        L.pic_get_particles.argtypes = [vp, C.c_int32, C.POINTER(pic_particles_view), C.c_int64]
        L.pic_set_particles.argtypes = [vp, C.c_int32, C.POINTER(pic_particles_view)]
        L.pic_set_step.argtypes = [vp, C.c_int64]
        L.pic_set_boundary.argtypes = [vp, vp, C.c_int32]
        L.pic_get_fields.argtypes = [vp] * 6 + [C.c_int32]
        L.pic_get_counts.argtypes = [vp, _i64p, _i64p, _u64p]
        L.pic_save.argtypes = [vp, C.c_char_p]
        L.pic_load.argtypes = [vp, C.c_char_p]
        L.pic_profile.argtypes = [vp, C.c_int32]
        L.pic_timings.argtypes = [vp, _dp, _i64p, _i64p, C.c_int32]
        L.pic_destroy.argtypes = [vp]
        L.pic_destroy.restype = None
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = C.c_char_p
        L.pic_field_solve_noalloc.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_int32,
                                              C.c_int32, vp, vp, C.c_double, vp, vp, C.c_double,
                                              C.c_int32, vp, C.POINTER(pic_solve_info)]
        L.pic_status_string.argtypes = [C.c_int]
        L.pic_status_string.restype = C.c_char_p
        for name in SYMBOLS:
            if name not in ("pic_destroy", "pic_last_error", "pic_status_string"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


class Handle:
    """An initialised reactor (owns the C handle and the arrays it borrows)."""

    def __init__(self, ptr, cfg, keep):
        self.ptr = ptr
        self.cfg = cfg
        self._keep = keep
        self.nz, self.nr = cfg["nz"], cfg["nr"]

    def __del__(self):
        try:
            pic_destroy(self)
        except Exception:
            pass


def _check(h, st, hard=(PIC_ERR_ARG, PIC_ERR_CAPACITY, PIC_ERR_CUDA, PIC_ERR_STATE,
                        PIC_ERR_TIMEOUT)):
    if st in hard:
        msg = lib().pic_last_error(h.ptr if isinstance(h, Handle) else None)
        raise PicError(st, (msg or b"").decode() or lib().pic_status_string(st).decode())
    return st


def _torch_hooks():
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, ctx, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
        except Exception:
            return None

    def _free(ptr, nbytes, ctx, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(_alloc), FREE_FN(_free)


def pic_init(cfg: dict, load: bool = True, stream=None, torch_memory: bool = True) -> Handle:
    """Create a reactor from a workload dict (see workloads.config)."""
    L = lib()
    keep = []
    c = pic_config()
    c.mesh = pic_mesh(cfg["R"], cfg["L"], cfg["nz"], cfg["nr"])
    for s, sp in enumerate(cfg["species"]):
        c.sp[s] = pic_species(sp["q"], sp["m"], sp["n0"], sp["T_eV"], int(sp["n_init"]),
                              int(sp["capacity"]))
        xs = cfg["xsec"][s]
        sig = _d(xs["sigma"]).reshape(-1)
        thr = _d(xs["threshold"])
        kind = np.ascontiguousarray([KIND[k] if isinstance(k, str) else k for k in xs["kind"]],
                                    dtype=np.int32)
        keep += [sig, thr, kind]
        c.xs[s] = pic_xsec(int(xs["n_e"]), float(xs["E_max"]), len(kind), _p(sig), _p(thr),
                           _p(kind, _ip), float(xs.get("B_eV", 10.0)))
    amp, freq, ph = (_d(cfg["rf"][k]) for k in ("amp", "freq", "phase"))
    keep += [amp, freq, ph]
    c.rf = pic_rf(len(amp), _p(amp), _p(freq), _p(ph))
    g = cfg["gas"]
    c.gas = pic_gas(g["p_Pa"], g["T_K"], g["m_gas"])
    c.dt = cfg["dt"]
    c.seed = cfg["seed"]
    c.precision = {"fp64": PIC_FP64, "mixed": PIC_MIXED}[cfg.get("precision", "fp64")]
    c.weighting = {"zr2": 0, "zr": 1}[cfg.get("weighting", "zr2")]
    c.chi_face = {"max": 0, "mean": 1}[cfg.get("chi_face", "max")]
    c.scatter = {"vs": 0, "isotropic": 1}[cfg.get("scatter", "vs")]
    c.split_every = int(cfg.get("split_every", 0))
    c.mg_max_cycles = int(cfg.get("mg_max_cycles", 50))
    c.mg_tol = float(cfg.get("mg_tol", 1e-10))
    if cfg.get("phi_zL") is not None:
        pz = _d(cfg["phi_zL"])
        keep.append(pz)
        c.phi_zL = _p(pz)
    c.births_capacity = int(cfg.get("births_capacity", 0))
    c.eedf_bins = int(cfg.get("eedf_bins", 0))
    c.eedf_emax_eV = float(cfg.get("eedf_emax", 100.0))
    c.load = 1 if load else 0
    if torch_memory or stream is None:
        import torch

        if not torch.cuda.is_available():
            raise PicError(PIC_ERR_CUDA, "no CUDA device")
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        if torch_memory:
            a, f = _torch_hooks()
            keep += [a, f]
            c.alloc, c.free = a, f
    c.stream = stream
    c.circuit_C = float(cfg.get("circuit_C", 0.0))
    c.pusher = {"local": 0, "xyz": 1}[cfg.get("pusher", "local")]
    c.ion_subcycle = int(cfg.get("ion_subcycle", 1))
    c.mg_guess = {"previous": 0, "linear": 1}[cfg.get("mg_guess", "linear")]
    ptr = C.c_void_p()
    st = L.pic_init(C.byref(c), C.byref(ptr))
    if st != PIC_OK:
        raise PicError(st, f"pic_init failed: {L.pic_status_string(st).decode()}")
    keep.append(c)
    return Handle(ptr, cfg, keep)


def pic_step(h: Handle, nsteps: int = 1) -> int:
    return _check(h, lib().pic_step(h.ptr, int(nsteps)))


class Batch:
    """Reactors stepped together (pic_batch_*); keeps its handles alive."""

    def __init__(self, handles, stream=None):
        self.handles = list(handles)
        arr = (C.c_void_p * len(self.handles))(*[h.ptr for h in self.handles])
        ptr = C.c_void_p()
        st = lib().pic_batch_init(arr, len(self.handles), stream, C.byref(ptr))
        if st != PIC_OK:
            raise PicError(st, f"pic_batch_init failed: {lib().pic_status_string(st).decode()}")
        self.ptr = ptr

    def step(self, nsteps: int = 1):
        """Advance every reactor; returns the per-reactor statuses (as pic_step's)."""
        sts = (C.c_int32 * len(self.handles))()
        lib().pic_batch_step(self.ptr, int(nsteps), sts)
        out = list(sts)
        for h, st in zip(self.handles, out):
            _check(h, st)
        return out

    def close(self):
        if getattr(self, "ptr", None):
            lib().pic_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        self.close()


def pic_get_circuit(h: Handle):
    """(electrode voltage, electrode charge, capacitor charge) after the last step."""
    out = np.zeros(3)
    _check(h, lib().pic_get_circuit(h.ptr, _p(out)))
    return tuple(out)


def pic_window(h: Handle, nsteps: int, ckpt: int, w, amp0: float, phi_zL=None, grad: bool = True):
    """The collisionless window from the handle's particles: (J, dJ/d amp0,
    dJ/d phi_zL) with grad, else (J, None, None).  w: (nz, nr) weights."""
    wv = _d(w).reshape(-1)
    pz = None if phi_zL is None else _d(phi_zL)
    J = np.zeros(1)
    dA = np.zeros(1)
    dP = np.zeros(h.nr)
    _check(h, lib().pic_window(h.ptr, int(nsteps), int(ckpt), _p(wv), float(amp0),
                               _p(pz) if pz is not None else None, 1 if grad else 0, _p(J),
                               _p(dA), _p(dP)))
    return (float(J[0]), float(dA[0]), dP) if grad else (float(J[0]), None, None)


def window_function():
    """torch.autograd.Function for J(amp0, phi_zL) of the collisionless window:
    the forward calls pic_window with the gradient, the backward returns it
    scaled by the incoming gradient.  Use as
    ``window_function().apply(amp0, phi_zL, h, w, nsteps, ckpt)`` with amp0 a
    0-d FP64 tensor and phi_zL an (nr,) FP64 tensor."""
    import torch

    class WindowJ(torch.autograd.Function):
        @staticmethod
        def forward(ctx, amp0, phi_zL, h, w, nsteps, ckpt):
            J, dA, dP = pic_window(h, nsteps, ckpt, w, float(amp0), phi_zL.detach().cpu().numpy(), True)
            ctx.save_for_backward(torch.tensor(dA, dtype=torch.float64),
                                  torch.as_tensor(dP, dtype=torch.float64))
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            dA, dP = ctx.saved_tensors
            return gJ * dA, gJ * dP.to(gJ.device), None, None, None, None

    return WindowJ


def pic_merge(h: Handle, s: int, frac: float, dv: float):
    """Merge the light particles of species s in pairs; (pairs, energy lost in J)."""
    n = C.c_int64(0)
    e = C.c_double(0)
    _check(h, lib().pic_merge(h.ptr, int(s), float(frac), float(dv), C.byref(n), C.byref(e)))
    return int(n.value), float(e.value)


def pic_selftest_wait(polls: int = 1 << 16) -> bool:
    """Run the bounded-wait self-test; True when the wait gave up as it must."""
    g = C.c_int32(0)
    st = lib().pic_selftest_wait(int(polls), C.byref(g))
    if st != PIC_OK:
        raise PicError(st, "pic_selftest_wait failed")
    return bool(g.value)


def pic_get_deposit(h: Handle):
    """The deposit the next solve takes: {"Ne", "Ni": [nz][nr], "q": [3]} (host)."""
    nz, nr = h.nz, h.nr
    Ne, Ni, q = np.zeros((nz, nr)), np.zeros((nz, nr)), np.zeros(3)
    _check(h, lib().pic_get_deposit(h.ptr, Ne.ctypes.data, Ni.ctypes.data, q.ctypes.data, 0))
    return {"Ne": Ne, "Ni": Ni, "q": q}


def pic_set_deposit(h: Handle, Ne, Ni, q=None) -> None:
    """Replace the deposit the next solve takes (host arrays)."""
    Ne = np.ascontiguousarray(Ne, dtype=np.float64)
    Ni = np.ascontiguousarray(Ni, dtype=np.float64)
    assert Ne.size == h.nz * h.nr and Ni.size == h.nz * h.nr
    qa = np.ascontiguousarray(q, dtype=np.float64) if q is not None else None
    _check(h, lib().pic_set_deposit(h.ptr, Ne.ctypes.data, Ni.ctypes.data,
                                    qa.ctypes.data if qa is not None else None, 0))


def pic_set_id_stride(h: Handle, next_id, stride: int) -> None:
    """Newborns of species s get ids next_id[s] + stride x rank (shared reactors)."""
    ids = (C.c_uint64 * 2)(*[int(x) for x in next_id])
    _check(h, lib().pic_set_id_stride(h.ptr, ids, int(stride)))


def pic_fp64_fma_rate(iters: int = 4096) -> float:
    """Measured FP64 fused multiply-add rate of the current device, GFLOP/s."""
    g = C.c_double(0.0)
    st = lib().pic_fp64_fma_rate(int(iters), C.byref(g))
    if st != PIC_OK:
        raise PicError(st, "pic_fp64_fma_rate failed")
    return g.value


def pic_tune(h: Handle, steps_per_variant: int = 2, variants=None):
    """Time the particle-pass shapes (or set them when steps_per_variant is 0);
    returns the shapes in use [electrons, ions]."""
    v = (C.c_int32 * 2)(*(variants if variants is not None else (-1, -1)))
    _check(h, lib().pic_tune(h.ptr, int(steps_per_variant), v))
    return list(v)


def pic_batch_init(handles, stream=None) -> Batch:
    return Batch(handles, stream)


def pic_batch_step(b: Batch, nsteps: int = 1):
    return b.step(nsteps)


def pic_batch_destroy(b: Batch) -> None:
    b.close()


def pic_field_solve(h: Handle, rho, chi, V: float):
    """Stand-alone solve on host arrays: returns (phi, cycles, rel_residual, status)."""
    rho, chi = _d(rho), _d(chi)
    phi = np.zeros((h.nz, h.nr))
    info = pic_solve_info()
    st = lib().pic_field_solve(h.ptr, rho.ctypes.data, chi.ctypes.data, float(V), phi.ctypes.data,
                               0, C.byref(info))
    _check(h, st)
    return phi, info.cycles, info.rel_residual, st


def pic_field_solve_device(h: Handle, rho_ptr: int, chi_ptr: int, V: float, phi_ptr: int):
    info = pic_solve_info()
    st = lib().pic_field_solve(h.ptr, rho_ptr, chi_ptr, float(V), phi_ptr, 1, C.byref(info))
    _check(h, st)
    return info.cycles, info.rel_residual, st


def pic_field_solve_noalloc(R: float, L: float, nz: int, nr: int, chi_face: int, rho_ptr: int,
                            chi_ptr: int, V: float, phi_zL_ptr, phi_ptr: int, tol: float,
                            max_cycles: int, stream=None):
    """Handle-free FP64 solve on device arrays that allocates no device memory (for
    callers that cannot allocate, e.g. during stream capture).  Returns
    (status, cycles, rel_residual); never raises, so callers can test the status."""
    info = pic_solve_info()
    st = lib().pic_field_solve_noalloc(float(R), float(L), int(nz), int(nr), int(chi_face),
                                       rho_ptr, chi_ptr, float(V), phi_zL_ptr, phi_ptr,
                                       float(tol), int(max_cycles), stream, C.byref(info))
    return st, info.cycles, info.rel_residual


def pic_moments(h: Handle, reset: bool = False) -> dict:
    nz, nr = h.nz, h.nr
    g = {k: np.zeros((nz, nr)) for k in ("ne", "ni", "phi", "Er", "Ez")}
    nb = max(int(h.cfg.get("eedf_bins", 0)), 1)
    eedf = np.zeros(nb)
    cnt = np.zeros(PIC_NCOUNT, dtype=np.int64)
    q = np.zeros(3)
    out = pic_moments_out(_p(g["ne"]), _p(g["ni"]), _p(g["phi"]), _p(g["Er"]), _p(g["Ez"]),
                          _p(eedf), _p(cnt, _i64p), _p(q), 0, 0)
    _check(h, lib().pic_moments(h.ptr, C.byref(out), 1 if reset else 0))
    g["eedf"] = eedf[: int(h.cfg.get("eedf_bins", 0))]
    g["counters"] = cnt
    g["charge"] = q
    g["nsamples"] = out.nsamples
    return g


def pic_moments_into(h: Handle, out: pic_moments_out, reset: bool = False) -> int:
    """Moments into caller-built buffers (host or device)."""
    return _check(h, lib().pic_moments(h.ptr, C.byref(out), 1 if reset else 0))


FIELDS = ("r", "z", "vr", "vt", "vz", "ar", "az", "w")


def pic_get_particles(h: Handle, s: int) -> dict:
    n = int(pic_get_counts(h)["n_alive"][s])
    arr = {k: np.zeros(n) for k in FIELDS}
    ids = np.zeros(n, dtype=np.uint64)
    cell = np.zeros(n, dtype=np.int32)
    at = np.zeros(n)
    v = pic_particles_view(n, *[_p(arr[k]) for k in FIELDS], _p(ids, _u64p), _p(cell, _ip), _p(at))
    _check(h, lib().pic_get_particles(h.ptr, s, C.byref(v), n))
    arr["id"] = ids[: v.n]
    arr["cell"] = cell[: v.n]
    arr["at"] = at[: v.n]
    for k in FIELDS:
        arr[k] = arr[k][: v.n]
    return arr


def pic_set_particles(h: Handle, s: int, p: dict) -> int:
    n = len(p["r"])
    arrs = [_d(p[k]) for k in FIELDS]
    ids = np.ascontiguousarray(p["id"], dtype=np.uint64)
    at = _d(p["at"]) if p.get("at") is not None else None
    v = pic_particles_view(n, *[_p(a) for a in arrs], _p(ids, _u64p), None,
                           _p(at) if at is not None else None)
    return _check(h, lib().pic_set_particles(h.ptr, s, C.byref(v)))


def pic_set_step(h: Handle, step: int) -> int:
    return _check(h, lib().pic_set_step(h.ptr, int(step)))


def pic_set_boundary(h: Handle, phi_zL, on_device: bool = False) -> int:
    if phi_zL is None:
        return _check(h, lib().pic_set_boundary(h.ptr, None, 0))
    if on_device:
        return _check(h, lib().pic_set_boundary(h.ptr, int(phi_zL), 1))
    a = _d(phi_zL)
    return _check(h, lib().pic_set_boundary(h.ptr, a.ctypes.data, 0))


def pic_get_fields(h: Handle) -> dict:
    g = {k: np.zeros((h.nz, h.nr)) for k in ("rho", "chi", "phi", "Ez", "Er")}
    _check(h, lib().pic_get_fields(h.ptr, *[g[k].ctypes.data for k in ("rho", "chi", "phi", "Ez", "Er")], 0))
    return g


def pic_get_counts(h: Handle) -> dict:
    n = np.zeros(2, dtype=np.int64)
    step = np.zeros(1, dtype=np.int64)
    nid = np.zeros(2, dtype=np.uint64)
    _check(h, lib().pic_get_counts(h.ptr, _p(n, _i64p), _p(step, _i64p), _p(nid, _u64p)))
    return dict(n_alive=n, step=int(step[0]), next_id=nid)


def pic_save(h: Handle, path: str) -> int:
    return _check(h, lib().pic_save(h.ptr, path.encode()))


def pic_load(h: Handle, path: str) -> int:
    return _check(h, lib().pic_load(h.ptr, path.encode()))


def pic_profile(h: Handle, on: bool = True) -> int:
    return _check(h, lib().pic_profile(h.ptr, 1 if on else 0))


def pic_timings(h: Handle, reset: bool = False) -> dict:
    ms = np.zeros(N_TIMING)
    pl = np.zeros(1, dtype=np.int64)
    al = np.zeros(1, dtype=np.int64)
    _check(h, lib().pic_timings(h.ptr, _p(ms), _p(pl, _i64p), _p(al, _i64p), 1 if reset else 0))
    return dict(solve_ms=ms[0], particle_e_ms=ms[1], particle_i_ms=ms[2], sort_ms=ms[3],
                other_ms=ms[4], particle_launches=int(pl[0]), launches=int(al[0]))


def pic_destroy(h: Handle) -> None:
    if getattr(h, "ptr", None):
        lib().pic_destroy(h.ptr)
        h.ptr = None


def pic_last_error(h: Handle) -> str:
    return (lib().pic_last_error(h.ptr) or b"").decode()
