"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 path 1e-12 relative per step, mixed FP32/FP64 path 2e-5,
for every particle and quantity element by element (tests/parity.py states
the floors), and for rho and chi node by node (relative to the node's charge
magnitude sum_s |q_s| N_s / V, resp. chi itself).  The potential and E are
compared in the max norm, the norm the field solve's stopping rule and
error bound are stated in.  Integer work is bit-exact in FP64 (cells, ids,
the cell-sort permutation's order and coverage, collision and split counts,
absorbed counts); in the mixed path an integer decision may differ only
where FP32 rounding of the inputs crosses the threshold, which each such
particle must show (parity.explain).
"""
import numpy as np
import pytest

import parity as P
import workloads as W
from oracle import C_ABS, C_BIRTHS, C_CAND, C_COLL, C_SPLITS, Oracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 2e-5}
FIELDS = ("r", "z", "vr", "vt", "vz", "ar", "az", "w")


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic as P

    build()
    return P


def by_id(p):
    o = np.argsort(p["id"], kind="stable")
    return {k: np.asarray(v)[o] for k, v in p.items()}


def nerr(a, b):
    """max |a - b| normalised by max |b| (0 when both vanish)."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    if a.size == 0:
        return 0.0
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a).max())


def cells_of(cfg, p):
    dz = cfg["L"] / (cfg["nz"] - 1)
    dr = cfg["R"] / (cfg["nr"] - 1)
    i = np.clip(np.floor(p["z"] / dz).astype(np.int64), 0, cfg["nz"] - 2)
    j = np.clip(np.floor(p["r"] / dr).astype(np.int64), 0, cfg["nr"] - 2)
    return j * (cfg["nz"] - 1) + i


def grid_node_errors(g, o, floor):
    """max over nodes of |g - o| / max(|o|, floor) (0 where both vanish)."""
    den = np.maximum(np.abs(o), floor)
    with np.errstate(invalid="ignore", divide="ignore"):
        e = np.where(den > 0, np.abs(g - o) / np.where(den > 0, den, 1.0), np.abs(g - o))
    return float(e.max(initial=0.0))


def make_pair(pic, cfg, load=True, capacity=None):
    o = Oracle(cfg, capacity=capacity)
    if load:
        o.load()
    h = pic.pic_init(cfg, load=load)
    return h, o


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_load_parity(pic, prec):
    cfg = W.config("c1", precision=prec)
    h, o = make_pair(pic, cfg)
    for s in (0, 1):
        g = pic.pic_get_particles(h, s)
        ref = o.get_particles(s)
        assert len(g["id"]) == len(ref["id"])
        # the load's cell of particle p follows from integer arithmetic alone
        n = cfg["species"][s]["n_init"]
        ncell = (cfg["nz"] - 1) * (cfg["nr"] - 1)
        base, rem = divmod(n, ncell)
        p = np.arange(n)
        c = np.where(p < rem * (base + 1), p // (base + 1), rem + (p - rem * (base + 1)) // max(base, 1))
        gs = by_id(g)
        assert np.array_equal(gs["cell"], c)
        P.check_sorted(g, (cfg["nz"] - 1) * (cfg["nr"] - 1))
        rs = by_id(ref)
        assert np.array_equal(gs["id"], rs["id"])
        # the loaded state: FP64 to 1e-12 (a position stored as cell + offset
        # is rounded to eps |x|, eps (nr - 1) of a cell width); mixed, one FP32
        # rounding of the cell offset, the velocities and the weight
        e = P.errors(cfg, s, gs, rs, 0.0, P.w_ref_table(cfg, s))
        assert e.max() <= (1e-12 if prec == "fp64" else 2e-7), float(e.max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_deposit_parity_after_load(pic, prec):
    cfg = W.config("c1", precision=prec)
    h, o = make_pair(pic, cfg)
    o.finalize()
    f = pic.pic_get_fields(h)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert nerr(f["rho"], o.grid("rho")) < tol
    assert nerr(f["chi"], o.grid("chi")) < tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mesh", [(33, 65), (65, 257), (129, 513)])
def test_field_solve_parity(pic, prec, mesh):
    nz, nr = mesh
    # the mixed path (FP32 V-cycles in FP64 refinement, GCR-accelerated) to a
    # relative residual of 1e-12, the oracle's plain V(0,1) to 1e-13: both
    # are then within ~cond(A) 1e-12 of the same discrete solution
    cfg = W.config("c1", nz=nz, nr=nr, precision=prec, mg_tol=1e-13 if prec == "fp64" else 1e-12,
                   mg_max_cycles=100)
    cfg = W.scaled(cfg, 0)
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    chi = W.random_grid(cfg, seed=nz, scale=2.0)
    rho = 1e-5 * (W.random_grid(cfg, seed=nr, smooth=False) - 0.5)
    phi, cyc, res, st = pic.pic_field_solve(h, rho, chi, 80.0)
    o.set_grid("chi", chi)
    o.set_grid("rho", rho)
    o.set_grid("phi", np.zeros((nz, nr)))
    ost, ocyc, ores = o.solve(80.0, tol=1e-13)
    assert st == 0 and ost == 0
    assert nerr(phi, o.grid("phi")) < (1e-12 if prec == "fp64" else 1e-9)
    if prec == "fp64":
        assert abs(cyc - ocyc) <= 1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_field_solve_single_interior_row(pic, prec):
    """nz = 3: one level, one interior row; the solve is one exact line solve.  (The
    r couplings of this row are ~160x its z couplings, so rounding leaves a relative
    residual near 1e-13: the tolerance sits above that floor.)"""
    cfg = W.scaled(W.config("c1", nz=3, nr=65, precision=prec, mg_tol=1e-11), 0)
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    chi = W.random_grid(cfg, seed=4, scale=1.5)
    rho = 1e-5 * (W.random_grid(cfg, seed=5, smooth=False) - 0.5)
    phi, cyc, res, st = pic.pic_field_solve(h, rho, chi, 25.0)
    o.set_grid("chi", chi)
    o.set_grid("rho", rho)
    o.set_grid("phi", np.zeros((3, 65)))
    ost, ocyc, _ = o.solve(25.0)
    assert st == 0 and ost == 0 and cyc == ocyc == 1
    assert nerr(phi, o.grid("phi")) < 1e-12


@pytest.mark.parametrize("cycles", [1, 3])
def test_field_solve_fixed_cycles_fp64_iterates(pic, cycles):
    """Same V-cycle, same number of cycles: the FP64 iterates agree to rounding."""
    cfg = W.scaled(W.config("c1", nz=65, nr=129, mg_tol=0.0, mg_max_cycles=cycles), 0)
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    chi = W.random_grid(cfg, seed=1, scale=1.0)
    rho = 1e-5 * (W.random_grid(cfg, seed=2, smooth=False) - 0.5)
    phi, cyc, res, st = pic.pic_field_solve(h, rho, chi, -40.0)
    o.set_grid("chi", chi)
    o.set_grid("rho", rho)
    o.set_grid("phi", np.zeros((65, 129)))
    o.solve(-40.0, tol=0.0, max_cycles=cycles)
    assert cyc == cycles
    assert nerr(phi, o.grid("phi")) < 1e-13


def _state_cfg(prec, capacity=400_000, **kw):
    """c1 geometry, no load (n_init 0: one reference particle per cell), room for `capacity`."""
    cfg = W.config("c1", precision=prec, **kw)
    for sp in cfg["species"]:
        sp["n_init"] = 0
        sp["capacity"] = capacity
    return cfg


def _random_state(cfg, n_e, n_i, seed, hot=3.0):
    e = W.random_particles(cfg, 0, n_e, seed=seed, hot=hot, accel=2e14, wscale=1.5e6)
    i = W.random_particles(cfg, 1, n_i, seed=seed + 1, hot=30.0, accel=5e9, wscale=1.5e6)
    return e, i


def _counters_match(gc, oc, prec):
    idx = list(range(C_COLL, C_COLL + 8)) + [C_CAND, C_CAND + 1] + [C_BIRTHS, C_BIRTHS + 1] + \
        [C_SPLITS, C_SPLITS + 1] + list(range(C_ABS, C_ABS + 6))
    for k in idx:
        if prec == "fp64":
            assert gc[k] == oc[k], (k, gc[k], oc[k])
        else:
            assert abs(int(gc[k]) - int(oc[k])) <= max(3, 1e-4 * oc[k]), (k, gc[k], oc[k])


def _one_step(pic, cfg, e, i, step_index, prec):
    h = pic.pic_init(cfg, load=False)
    o = Oracle(cfg)
    pic.pic_set_particles(h, 0, e)
    pic.pic_set_particles(h, 1, i)
    o.set_particles(0, e)
    o.set_particles(1, i)
    pic.pic_set_step(h, step_index)
    o.set_step(step_index)
    st = pic.pic_step(h, 1)
    o.step(1)
    assert st == 0
    f = pic.pic_get_fields(h)
    grids = {k: o.grid(k) for k in ("phi", "Ez", "Er")}
    o.finalize()
    tol = TOL[prec]
    for name in ("phi", "Ez", "Er"):
        assert nerr(f[name], grids[name]) < (tol if prec == "fp64" else 1e-6), name
    # rho and chi node by node, relative to the node's charge magnitude
    # (electron and ion charge cancel where the plasma is neutral) plus what
    # one particle of the split's reference weight adds there (a node that a
    # single particle barely reaches holds a tiny, rounding-sized value)
    V = o.node_volumes()
    q, m = abs(cfg["species"][0]["q"]), cfg["species"][0]["m"]
    w1 = P.w_ref_table(cfg, 0)[np.minimum(np.arange(cfg["nr"]), cfg["nr"] - 2)][None, :] / V
    qabs = q * ((o.grid("Ne") + o.grid("Ni")) / V + w1)
    chi1 = q * q / m * w1 * cfg["dt"] ** 2 / (2.0 * 8.8541878128e-12)
    assert grid_node_errors(f["rho"], o.grid("rho"), qabs) <= tol
    assert grid_node_errors(f["chi"], o.grid("chi"), chi1) <= tol
    explained = 0
    for s, inp in ((0, e), (1, i)):
        g = pic.pic_get_particles(h, s)
        ref = o.get_particles(s)
        explained += P.compare_species(cfg, s, g, ref, prec, inputs=inp, grids=grids, step=step_index)
    m = pic.pic_moments(h)
    oc, oq = o.counters()
    _counters_match(m["counters"], oc, prec)
    assert nerr(m["charge"], oq) < (1e-12 if prec == "fp64" else 1e-4)
    cnt = pic.pic_get_counts(h)
    if prec == "fp64":
        assert list(cnt["next_id"]) == [o.next_id(0), o.next_id(1)]
    return h, o, oc


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_one_step_parity_with_collisions_and_births(pic, prec):
    cfg = _state_cfg(prec)
    e, i = _random_state(cfg, 60_001, 40_003, seed=5)
    h, o, oc = _one_step(pic, cfg, e, i, 17, prec)
    assert oc[C_COLL + 2] > 50  # ionisations happened
    assert oc[C_COLL + 4] > 0  # charge exchange happened
    assert oc[C_ABS:C_ABS + 6].sum() > 0  # walls absorbed


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_one_step_parity_with_splitting(pic, prec):
    cfg = _state_cfg(prec, split_every=1)
    e, i = _random_state(cfg, 20_000, 20_000, seed=9, hot=1.0)
    o = Oracle(cfg)
    dr = cfg["R"] / (cfg["nr"] - 1)
    rng = np.random.default_rng(3)
    for p, s in ((e, 0), (i, 1)):
        j = np.minimum(np.floor(p["r"] / dr).astype(int), cfg["nr"] - 2)
        wr = np.array([o.w_ref(s, int(k)) for k in j])
        p["w"] = wr * rng.uniform(0.3, 12.0, len(j))
    h, o2, oc = _one_step(pic, cfg, e, i, 0, prec)
    assert oc[C_SPLITS] > 1000 and oc[C_SPLITS + 1] > 1000


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tiny_and_empty_inputs(pic, prec):
    cfg = W.config("tiny", precision=prec)
    rng = np.random.default_rng(0)
    e = W.random_particles(cfg, 0, 7, seed=1, hot=4.0)
    i = W.random_particles(cfg, 1, 0, seed=2)
    _one_step(pic, cfg, e, i, 3, prec)
    # both species empty: the field is the vacuum (Laplace) solution
    cfg2 = W.config("tiny", precision=prec)
    h = pic.pic_init(W.scaled(cfg2, 0), load=False)
    assert pic.pic_step(h, 2) == 0
    assert list(pic.pic_get_counts(h)["n_alive"]) == [0, 0]


@pytest.mark.parametrize("guess", ["linear", "previous"])
def test_multi_step_parity_fp64(pic, guess):
    """Five steps: the FP64 path runs the oracle's V-cycle iterates, from the
    same starting value (the last potential, or its linear extrapolation from
    the last two steps), so the cycle counts agree step by step."""
    cfg = W.scaled(W.config("c1", precision="fp64", mg_guess=guess), 20_000)
    h, o = make_pair(pic, cfg)
    K = 5
    ocyc = 0
    for _ in range(K):
        pic.pic_step(h, 1)
        ocyc += o.step(1)[0]
    f = pic.pic_get_fields(h)
    for name in ("phi", "Ez", "Er"):
        assert nerr(f[name], o.grid(name)) < 1e-11, name
    for s in (0, 1):
        g = by_id(pic.pic_get_particles(h, s))
        ref = by_id(o.get_particles(s))
        assert np.array_equal(g["id"], ref["id"])
        for k in FIELDS:
            assert nerr(g[k], ref[k]) < 1e-10, k
    m = pic.pic_moments(h)
    oc, _ = o.counters()
    _counters_match(m["counters"], oc, "fp64")
    assert int(m["counters"][pic.PIC_C_MGCYC]) == ocyc
    om = o.moments()
    for k in ("ne", "ni", "phi", "Ez", "Er"):
        assert nerr(m[k], om[k]) < 1e-10, k
    assert nerr(m["eedf"], om["eedf"]) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(pic, prec):
    """Steps replayed as CUDA graphs (the default) give what the same steps
    launched one by one (profiling on) give: the same ids, counts and
    counters, fields and particles to rounding (deposit atomics add in any
    order).  Five steps in two calls cover both buffer parities."""
    cfg = W.scaled(W.config("c1", precision=prec), 20_000)
    ha, hb = pic.pic_init(cfg), pic.pic_init(cfg)
    pic.pic_profile(ha, True)
    for k in (3, 2):
        assert pic.pic_step(ha, k) == 0
        assert pic.pic_step(hb, k) == 0
    ca, cb = pic.pic_get_counts(ha), pic.pic_get_counts(hb)
    assert ca["step"] == cb["step"] == 5
    tol = 1e-11 if prec == "fp64" else 1e-5
    fa, fb = pic.pic_get_fields(ha), pic.pic_get_fields(hb)
    for name in ("phi", "rho", "Ez"):
        assert nerr(fb[name], fa[name]) < tol, name
    for s in (0, 1):
        ga, gb = by_id(pic.pic_get_particles(ha, s)), by_id(pic.pic_get_particles(hb, s))
        if prec == "fp64":
            assert np.array_equal(ga["id"], gb["id"])
            assert list(ca["next_id"]) == list(cb["next_id"])
            for k in FIELDS:
                assert nerr(gb[k], ga[k]) < 1e-10, k
        else:
            common = np.intersect1d(ga["id"], gb["id"])
            assert len(common) >= len(ga["id"]) - 5
    ma, mb = pic.pic_moments(ha), pic.pic_moments(hb)
    if prec == "fp64":
        assert list(ma["counters"][:22]) == list(mb["counters"][:22])
    assert ma["counters"][pic.PIC_C_STEPS] == mb["counters"][pic.PIC_C_STEPS] == 5


def test_births_capacity_error_keeps_the_state(pic):
    cfg = _state_cfg("fp64", births_capacity=16)
    e, i = _random_state(cfg, 30_000, 1000, seed=21, hot=4.0)
    h = pic.pic_init(cfg, load=False)
    pic.pic_set_particles(h, 0, e)
    pic.pic_set_particles(h, 1, i)
    before = by_id(pic.pic_get_particles(h, 0))
    with pytest.raises(pic.PicError) as err:
        pic.pic_step(h, 1)
    assert err.value.status == pic.PIC_ERR_CAPACITY
    after = by_id(pic.pic_get_particles(h, 0))
    for k in FIELDS + ("id",):
        assert np.array_equal(before[k], after[k])


@pytest.mark.parametrize("variant", ["zr", "mean", "isotropic", "phi_zL"])
def test_one_step_parity_variants(pic, variant):
    """The flags of the paper's alternatives (Sec. 2.4 z-r weighting, Sec. 2.5 mean face
    rule) and of the test scattering law, and Dirichlet data on z = L."""
    kw = {"zr": dict(weighting="zr"), "mean": dict(chi_face="mean"),
          "isotropic": dict(scatter="isotropic"), "phi_zL": {}}[variant]
    cfg = _state_cfg("fp64", **kw)
    if variant == "phi_zL":
        cfg["phi_zL"] = 20.0 * np.cos(np.linspace(0, np.pi / 2, cfg["nr"]))
    e, i = _random_state(cfg, 30_000, 20_000, seed=31)
    _one_step(pic, cfg, e, i, 5, "fp64")


def test_checkpoint_resume_matches_uninterrupted_run(pic, tmp_path):
    cfg = W.scaled(W.config("c1", precision="fp64"), 20_000)
    h1 = pic.pic_init(cfg)
    pic.pic_step(h1, 3)
    path = str(tmp_path / "ck.bin")
    pic.pic_save(h1, path)
    h2 = pic.pic_init(cfg, load=False)
    pic.pic_load(h2, path)
    assert pic.pic_get_counts(h2)["step"] == 3
    pic.pic_step(h1, 2)
    pic.pic_step(h2, 2)
    for s in (0, 1):
        a, b = by_id(pic.pic_get_particles(h1, s)), by_id(pic.pic_get_particles(h2, s))
        assert np.array_equal(a["id"], b["id"])
        for k in FIELDS:
            assert nerr(b[k], a[k]) < 1e-12, k
    fa, fb = pic.pic_get_fields(h1), pic.pic_get_fields(h2)
    assert nerr(fb["phi"], fa["phi"]) < 1e-12


def test_particle_capacity_error_keeps_the_state(pic):
    cfg = _state_cfg("fp64", capacity=30_050, split_every=1)
    e, i = _random_state(cfg, 30_000, 1000, seed=41, hot=1.0)
    o = Oracle(cfg)
    dr = cfg["R"] / (cfg["nr"] - 1)
    j = np.minimum(np.floor(e["r"] / dr).astype(int), cfg["nr"] - 2)
    e["w"] = np.array([o.w_ref(0, int(k)) for k in j]) * 3.5  # every electron splits into 3-4
    h = pic.pic_init(cfg, load=False)
    pic.pic_set_particles(h, 0, e)
    pic.pic_set_particles(h, 1, i)
    before = by_id(pic.pic_get_particles(h, 0))
    with pytest.raises(pic.PicError) as err:
        pic.pic_step(h, 1)
    assert err.value.status == pic.PIC_ERR_CAPACITY
    after = by_id(pic.pic_get_particles(h, 0))
    for k in FIELDS + ("id",):
        assert np.array_equal(before[k], after[k])
    assert pic.pic_get_counts(h)["step"] == 0


def test_non_finite_particles_are_dropped_and_reported(pic):
    cfg = _state_cfg("fp64")
    e, i = _random_state(cfg, 1000, 1000, seed=51)
    e["vz"][7] = np.nan
    h = pic.pic_init(cfg, load=False)
    pic.pic_set_particles(h, 0, e)
    pic.pic_set_particles(h, 1, i)
    st = pic.pic_step(h, 1)
    assert st == pic.PIC_ERR_NUMERIC
    g = pic.pic_get_particles(h, 0)
    assert e["id"][7] not in set(g["id"].tolist())
    assert np.all(np.isfinite(g["vz"]))


def test_moments_into_device_buffers(pic):
    torch = pytest.importorskip("torch")
    import ctypes as C

    cfg = W.scaled(W.config("c1", precision="mixed"), 20_000)
    h = pic.pic_init(cfg)
    pic.pic_step(h, 3)
    host = pic.pic_moments(h)
    bufs = [torch.zeros(cfg["nz"] * cfg["nr"], dtype=torch.float64, device="cuda") for _ in range(5)]
    dp = C.POINTER(C.c_double)
    out = pic.pic_moments_out(*[C.cast(b.data_ptr(), dp) for b in bufs], None, None, None, 0, 1)
    pic.pic_moments_into(h, out)
    torch.cuda.synchronize()
    for name, b in zip(("ne", "ni", "phi", "Er", "Ez"), bufs):
        np.testing.assert_array_equal(b.cpu().numpy().reshape(cfg["nz"], cfg["nr"]), host[name])
    assert out.nsamples == 3
