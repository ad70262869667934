"""The allocation-free field solve against the handle's field solve.

pic_field_solve_noalloc serves callers that cannot allocate device memory
when they solve (a host that fixed the library's memory budget at start-up,
a real-time loop that must not stall on an allocation): it must give the
same potential as pic_field_solve, call after call, while using only its
fixed workspace -- the device's free memory does not change across a call.
On one mesh the reference is also checked against the FP64 oracle's solve.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic

    build()
    return torch, pic


def _nerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("mesh", [(65, 257), (129, 513), (33, 1025)])
def test_noalloc_solve_matches_handle_solve_on_two_calls_in_a_row(env, mesh):
    """(129, 513) is the largest mesh the workspace holds; (33, 1025) is a wide,
    short one whose line solves take more than 48 KB of shared memory."""
    torch, pic = env
    nz, nr = mesh
    cfg = W.scaled(W.config("c1", nz=nz, nr=nr, R=0.05 * (nr - 1) / 64, mg_tol=1e-12, mg_max_cycles=60), 0)
    h = pic.pic_init(cfg, load=False)
    stream = torch.cuda.current_stream().cuda_stream
    calls = []
    for seed, V, with_zL in ((11, 60.0, False), (12, -35.0, True)):
        chi = W.random_grid(cfg, seed=seed, scale=2.0)
        rho = 1e-5 * (W.random_grid(cfg, seed=seed + 100, smooth=False) - 0.5)
        zL = np.linspace(5.0, 0.0, nr) if with_zL else None
        pic.pic_set_boundary(h, zL)
        ref, cyc_ref, _, st_ref = pic.pic_field_solve(h, rho, chi, V)
        assert st_ref == pic.PIC_OK
        if mesh == (65, 257):
            # the handle's solve is the oracle's: the same V(0,1) iterates
            o = Oracle(dict(cfg, phi_zL=zL))
            o.set_grid("chi", chi)
            o.set_grid("rho", rho)
            o.set_grid("phi", np.zeros((nz, nr)))
            assert o.solve(V, tol=1e-12, max_cycles=60)[0] == 0
            assert _nerr(ref, o.grid("phi")) < 1e-12
        dev = dict(rho=torch.tensor(rho, dtype=torch.float64, device="cuda"),
                   chi=torch.tensor(chi, dtype=torch.float64, device="cuda"),
                   phi=torch.full((nz, nr), float("nan"), dtype=torch.float64, device="cuda"),
                   zL=torch.tensor(zL, dtype=torch.float64, device="cuda") if with_zL else None)
        calls.append((V, dev, ref, cyc_ref))
    pic.pic_destroy(h)
    torch.cuda.synchronize()
    free = []
    for V, dev, ref, cyc_ref in calls:
        free.append(torch.cuda.mem_get_info()[0])
        st, cyc, res = pic.pic_field_solve_noalloc(
            cfg["R"], cfg["L"], nz, nr, 0, dev["rho"].data_ptr(), dev["chi"].data_ptr(), V,
            dev["zL"].data_ptr() if dev["zL"] is not None else None, dev["phi"].data_ptr(), 1e-12, 60,
            stream)
        torch.cuda.synchronize()
        assert st == pic.PIC_OK, st
        assert cyc == cyc_ref and res <= 1e-12
        assert _nerr(dev["phi"].cpu().numpy(), ref) < 1e-12
    free.append(torch.cuda.mem_get_info()[0])
    # the second call (the first may load the module's kernels) leaves the
    # device's free memory as it found it
    assert free[2] == free[1], free


def test_noalloc_solve_rejects_a_mesh_beyond_its_workspace(env):
    torch, pic = env
    nz, nr = 257, 1025
    d = torch.zeros((nz, nr), dtype=torch.float64, device="cuda")
    st, _, _ = pic.pic_field_solve_noalloc(0.3, 0.03, nz, nr, 0, d.data_ptr(), d.data_ptr(), 1.0,
                                           None, d.data_ptr(), 1e-10, 10,
                                           torch.cuda.current_stream().cuda_stream)
    assert st == pic.PIC_ERR_ARG
