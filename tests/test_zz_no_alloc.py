"""The allocation-free field solve against the handle's field solve.

pic_field_solve_noalloc serves callers that cannot allocate device memory
when they solve (stream capture, fixed memory budgets, real-time loops): it
must give the same potential as pic_field_solve, call after call, while
using only its fixed workspace.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

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


def test_noalloc_solve_matches_handle_solve_on_two_calls_in_a_row(env):
    torch, pic = env
    nz, nr = 65, 257
    cfg = W.scaled(W.config("c1", nz=nz, nr=nr, mg_tol=1e-12, mg_max_cycles=60), 0)
    h = pic.pic_init(cfg, load=False)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (seed, V, with_zL) in enumerate(((11, 60.0, False), (12, -35.0, True))):
        chi = W.random_grid(cfg, seed=seed, scale=2.0)
        rho = 1e-5 * (W.random_grid(cfg, seed=seed + 100, smooth=False) - 0.5)
        zL = np.linspace(5.0, 0.0, nr) if with_zL else None
        pic.pic_set_boundary(h, zL)
        ref, cyc_ref, _, st_ref = pic.pic_field_solve(h, rho, chi, V)
        assert st_ref == pic.PIC_OK
        d_rho = torch.tensor(rho, dtype=torch.float64, device="cuda")
        d_chi = torch.tensor(chi, dtype=torch.float64, device="cuda")
        d_phi = torch.full((nz, nr), float("nan"), dtype=torch.float64, device="cuda")
        d_zL = torch.tensor(zL, dtype=torch.float64, device="cuda") if with_zL else None
        st, cyc, res = pic.pic_field_solve_noalloc(
            cfg["R"], cfg["L"], nz, nr, 0, d_rho.data_ptr(), d_chi.data_ptr(), V,
            d_zL.data_ptr() if with_zL else None, d_phi.data_ptr(), 1e-12, 60, stream)
        torch.cuda.synchronize()
        assert st == pic.PIC_OK, (call, st)
        assert cyc == cyc_ref and res <= 1e-12
        assert _nerr(d_phi.cpu().numpy(), ref) < 1e-12, call


def test_noalloc_solve_rejects_a_mesh_beyond_its_workspace(env):
    torch, pic = env
    nz, nr = 257, 1025
    d = torch.zeros((nz, nr), dtype=torch.float64, device="cuda")
    st, _, _ = pic.pic_field_solve_noalloc(0.3, 0.03, nz, nr, 0, d.data_ptr(), d.data_ptr(), 1.0,
                                           None, d.data_ptr(), 1e-10, 10,
                                           torch.cuda.current_stream().cuda_stream)
    assert st == pic.PIC_ERR_ARG
