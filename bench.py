#!/usr/bin/env python3
"""Throughput of the implicit r-z PIC/MC timestep on one GB300 (arXiv:1001.2969).

A step is one whole implicit timestep of the production-size reactor
(R 20 cm, L 2.5 cm, 129 x 513 nodes, 1e7 electrons + 1e7 Ar+, 300 V at
13.56 MHz, dt = T_rf/200): deposit -> multigrid solve -> E -> fused particle
pass (gather, push, MC, split, push, deposit) -> cell sort.  The metric is
particle-steps per second, mixed FP32/FP64 path, with the plain FP64 path
reported beside it.  Inputs (the particle state, 880 MB mixed) are larger
than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Under torchrun each rank runs its own reactor (independent replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and ms/step at 20M particles (mixed vs FP64); % of HBM peak"
UNIT = "particle-steps/s"
WORKLOADS = {
    "c2": ("c2 production reactor: R 20 cm, L 2.5 cm, 129x513 nodes, 1e7 e- + 1e7 Ar+, "
           "n0 5e15 m^-3, argon 4 Pa 300 K, 300 V at 13.56 MHz, dt = T_rf/200, seed 1"),
    "c1": ("c1 small reactor: R 5 cm, L 2 cm, 33x65 nodes, 1e5 e- + 1e5 Ar+, n0 1e15 m^-3, "
           "argon 4 Pa 300 K, 100 V at 13.56 MHz, dt = T_rf/400, seed 1"),
    "c3": ("c3 large dual-frequency reactor: R 30 cm, L 3 cm, 257x1025 nodes, 1e8 e- + 1e8 Ar+, "
           "n0 5e15 m^-3, argon 8 Pa 300 K, 200 V at 60 MHz + 500 V at 2 MHz, dt = T_60MHz/100, seed 1"),
}
WORKLOAD = WORKLOADS["c2"]
# algorithmic bytes of the particle pass per particle: the state read once and
# written once (mixed: cell 4 + offsets 8 + v 12 + a 8 + w 4 + id 8 = 44 B)
BYTES_PER_PARTICLE = {"mixed": 88, "fp64": 152}
# FP64 floating-point operations of the FP64 particle pass per particle-step
# (2 DFMA + DADD + DMUL thread instructions; ncu on the c2 mesh, 1M + 1M
# particles: electrons 256, ions 225; profiles/k_step_fp64_c2.md)
FP64_FLOPS_PER_PARTICLE = 240


def whole_job(ms, psteps, e2e_seconds, e2e_psteps, world, device="cuda"):
    """Whole-job figures over `world` ranks of independent replicas: the
    particle-steps all ranks processed over the slowest rank's time, for the
    device-timed region and for the end-to-end one.  Returns (ms_max,
    psteps_sum, e2e_seconds_max, e2e_psteps_sum); one rank returns its own."""
    if world <= 1:
        return ms, psteps, e2e_seconds, e2e_psteps
    import torch

    t_max = torch.tensor([ms, e2e_seconds], dtype=torch.float64, device=device)
    n_sum = torch.tensor([psteps, e2e_psteps], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t_max, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(n_sum, op=torch.distributed.ReduceOp.SUM)
    return float(t_max[0]), float(n_sum[0]), float(t_max[1]), float(n_sum[1])


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader",
                                       "-lms", "50", "-i", str(self.dev)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.strip() for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            c = [x.strip() for x in r.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1].split()[0]))
                mx.append(float(c[2].split()[0]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if c[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic(prec):
    """DRAM bytes per particle of the particle pass from the committed ncu summary."""
    p = os.path.join(ROOT, "profiles", f"k_step_{prec}_c2.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith("dram_bytes_per_particle:"):
            try:
                return float(line.split(":")[1])
            except ValueError:
                return None
    return None


def run_gpu(args, rank, world):
    import numpy as np
    import torch

    import workloads as W
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic

    build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    results = {}
    for prec in (args.precision, "fp64") if args.fp64_steps > 0 else (args.precision,):
        steps = args.steps if prec == args.precision else args.fp64_steps
        cfg = W.config(args.config, precision=prec, seed=1 + rank, ion_subcycle=args.ion_subcycle)
        if args.particles:
            cfg = W.scaled(cfg, args.particles)
        h = pic.pic_init(cfg, stream=stream.cuda_stream)
        statuses = [pic.pic_step(h, args.warmup)]
        n0 = pic.pic_get_counts(h)["n_alive"].sum()
        if world > 1:
            torch.distributed.barrier()
        pic.pic_moments(h, reset=True)  # restarts the V-cycle count
        torch.cuda.synchronize()
        clocks = Clocks(dev) if prec == args.precision else None
        if clocks:
            clocks.start()
        pic.pic_timings(h, reset=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = pic.pic_step(h, steps)  # each step one CUDA graph replay
        ev1.record(stream)
        statuses.append(st)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ck = clocks.stop() if clocks else None
        launches = pic.pic_timings(h, reset=True)["launches"]
        ms = ev0.elapsed_time(ev1)
        cnt = pic.pic_moments(h, reset=True)["counters"]
        cycles = int(cnt[pic.PIC_C_MGCYC])
        n1 = pic.pic_get_counts(h)["n_alive"].sum()
        # particles the passes moved, counted on the device step by step (the
        # count changes with losses, births and the periodic split)
        psteps = float(cnt[pic.PIC_C_PSTEPS])
        # phase breakdown and the particle kernel's own time: the same number of
        # steps again, launched one by one with CUDA events around each phase
        pic.pic_profile(h, True)
        statuses.append(pic.pic_step(h, steps))
        pic.pic_profile(h, False)
        tm = pic.pic_timings(h, reset=True)
        prof_psteps = float(pic.pic_moments(h, reset=True)["counters"][pic.PIC_C_PSTEPS])
        res = dict(ms=ms, psteps=psteps, prof_psteps=prof_psteps, n0=int(n0), n1=int(n1), timings=tm,
                   clocks=ck, status=st, statuses=statuses, mg_cycles=cycles / steps, launches=launches)
        if prec == args.precision:
            # end to end through the public API with host buffers: per step the z = L
            # boundary row goes host -> device from pinned memory and the time-averaged
            # grids come back device -> host
            phiL = torch.zeros(cfg["nr"], dtype=torch.float64, pin_memory=True)
            nz, nr = cfg["nz"], cfg["nr"]
            outs = [torch.zeros(nz * nr, dtype=torch.float64, pin_memory=True) for _ in range(5)]
            import ctypes as C

            mo = pic.pic_moments_out(*[C.cast(o.data_ptr(), C.POINTER(C.c_double)) for o in outs],
                                     None, None, None, 0, 0)
            e_steps = max(1, min(steps, args.e2e_steps))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e_steps):
                pic.lib().pic_set_boundary(h.ptr, phiL.data_ptr(), 0)
                statuses.append(pic.pic_step(h, 1))
                pic.pic_moments_into(h, mo)
            torch.cuda.synchronize()
            e2e_s = time.perf_counter() - t0
            e_ps = float(pic.pic_moments(h)["counters"][pic.PIC_C_PSTEPS])
            res["e2e"] = dict(seconds=e2e_s, psteps=e_ps, steps=e_steps, h2d=nr * 8, d2h=5 * nz * nr * 8)
        pic.pic_destroy(h)
        del h
        torch.cuda.empty_cache()
        results[prec] = res
    return results


def solve_only(args):
    """Time the stand-alone field solve (pic_field_solve on device arrays) on the
    workload's mesh with seeded random rho and chi, both precisions."""
    import torch

    import workloads as W
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic

    build()
    out = {}
    for prec in ("mixed", "fp64"):
        cfg = W.scaled(W.config(args.config, precision=prec), 0)
        h = pic.pic_init(cfg, load=False)
        chi = W.random_grid(cfg, seed=1, scale=1.0)
        rho = 1e-5 * (W.random_grid(cfg, seed=2, smooth=False) - 0.5)
        d_rho = torch.tensor(rho, device="cuda")
        d_chi = torch.tensor(chi, device="cuda")
        d_phi = torch.zeros_like(d_rho)
        pic.pic_field_solve_device(h, d_rho.data_ptr(), d_chi.data_ptr(), 100.0, d_phi.data_ptr())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            cyc, res, st = pic.pic_field_solve_device(h, d_rho.data_ptr(), d_chi.data_ptr(), 100.0,
                                                      d_phi.data_ptr())
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / max(args.steps, 1)
        out[prec] = {"ms_per_solve": dt * 1e3, "cycles": cyc, "rel_residual": res, "status": st}
        pic.pic_destroy(h)
    print(json.dumps({"solve_only": out, "config": args.config}))
    return 0


def cpu_baseline(cfg_name, n_per_species, steps):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload."""
    import workloads as W
    from oracle import Oracle

    cfg = W.scaled(W.config(cfg_name), n_per_species)
    o = Oracle(cfg)
    o.load()
    o.step(1)  # first step outside the timing (warm caches)
    n0 = o.count(0) + o.count(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    n1 = o.count(0) + o.count(1)
    ps = 0.5 * (n0 + n1) * steps
    return {"value": ps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{cfg_name} mesh and load with {n_per_species} particles per species "
                      f"(1/{int(W.config(cfg_name)['species'][0]['n_init'] / n_per_species)} of the "
                      f"workload), {steps} steps after one warm-up step, single thread",
            "ms_per_step": 1e3 * dt / steps}


def accuracy_vs_oracle(cfg_name, n_per_species, stream):
    """Each output's error against the FP64 oracle after one step of the same
    seeded sample of the workload (both GPU precisions): fields relative to
    their largest magnitude, particle states likewise over the particles both
    sides hold, and how many particles one side holds and the other not
    (FP32 decisions at thresholds)."""
    import numpy as np
    import workloads as W
    from oracle import Oracle
    from paper_1001_2969_gb300 import pic

    cfg = W.scaled(W.config(cfg_name), n_per_species)
    o = Oracle(cfg)
    o.load()
    o.step(1)
    o.finalize()
    ref_f = {k: o.grid(k) for k in ("phi", "Ez", "Er", "rho", "chi")}
    ref_p = [o.get_particles(s) for s in (0, 1)]
    out = {"sample": f"{cfg_name} mesh and load with {n_per_species} particles per species, one step",
           "norm": "max |gpu - oracle| / max |oracle| per output"}
    for prec in ("mixed", "fp64"):
        h = pic.pic_init(W.scaled(W.config(cfg_name, precision=prec), n_per_species),
                         stream=stream.cuda_stream)
        pic.pic_step(h, 1)
        f = pic.pic_get_fields(h)
        r = {k: float(np.abs(f[k] - ref_f[k]).max() / np.abs(ref_f[k]).max()) for k in ref_f}
        worst, unmatched = {}, 0
        for s in (0, 1):
            g = pic.pic_get_particles(h, s)
            common, gi, oi = np.intersect1d(g["id"], ref_p[s]["id"], return_indices=True)
            unmatched += len(g["id"]) + len(ref_p[s]["id"]) - 2 * len(common)
            for k in ("r", "z", "vr", "vt", "vz", "w"):
                a, b = np.asarray(g[k])[gi], np.asarray(ref_p[s][k])[oi]
                e = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
                worst[k] = max(worst.get(k, 0.0), e)
        r["particles"] = worst
        r["particles_on_one_side_only"] = int(unmatched)
        out[prec] = r
        pic.pic_destroy(h)
    return out


def batch_run(args):
    """The batched sweep: args.batch independent reactors (workloads.batch_configs),
    each tuned, then stepped together (one graph launch per step) and, for
    comparison, one after another; particle-steps/s over all reactors."""
    import torch
    import workloads as W
    from paper_1001_2969_gb300 import pic

    stream = torch.cuda.current_stream()
    cfgs = W.batch_configs(n=args.batch, precision=args.precision)
    t0 = time.perf_counter()
    hs = [pic.pic_init(c, stream=stream.cuda_stream) for c in cfgs]
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    shapes = [pic.pic_tune(h, 1) for h in hs]
    t_tune = time.perf_counter() - t0
    b = pic.pic_batch_init(hs, stream.cuda_stream)
    b.step(args.warmup)

    def count():
        return sum(int(pic.pic_get_counts(h)["n_alive"].sum()) for h in hs)

    def timed(fn):
        for h in hs:
            pic.pic_moments(h, reset=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ps = sum(float(pic.pic_moments(h)["counters"][pic.PIC_C_PSTEPS]) for h in hs)
        return ps / (ms * 1e-3), ms / args.steps

    v_batch, ms_batch = timed(lambda: b.step(args.steps))

    def one_by_one():
        for _ in range(args.steps):
            for h in hs:
                pic.pic_step(h, 1)

    v_seq, ms_seq = timed(one_by_one)
    b.close()
    line = {"metric": "particle-steps/s of a batch of independent reactors", "unit": UNIT,
            "value": v_batch, "ms_per_step": ms_batch, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.batch} reactors drawn by workloads.batch_configs (seed 4): "
                                   "33x65 to 129x513 nodes, 5e4-5e6 particles per species, "
                                   "1-100 Pa, 50-500 V at 13.56 MHz",
                       "particles": count(), "precision": args.precision},
            "one_reactor_after_another": {"value": v_seq, "ms_per_step": ms_seq},
            "tuned_shapes": {"electrons": [s[0] for s in shapes], "ions": [s[1] for s in shapes]},
            "init_s": t_init, "tune_s": t_tune}
    print(json.dumps(line))
    return 0


def adjoint_run(args):
    """The adjoint window (workload c5): J alone and J with its gradient
    (rf amplitude, z = L row) from the loaded state, ms per call, and the
    forward's particle-steps/s."""
    import torch
    import workloads as W
    from paper_1001_2969_gb300 import pic

    stream = torch.cuda.current_stream()
    cfg = W.config("c5", precision=args.precision)
    if args.particles:
        cfg = W.scaled(cfg, args.particles)
    K, ck = cfg["steps"], cfg["ckpt"]
    w = W.gaussian_weight(cfg)
    amp = cfg["rf"]["amp"][0]
    h = pic.pic_init(cfg, stream=stream.cuda_stream)
    n = int(pic.pic_get_counts(h)["n_alive"].sum())
    pic.pic_window(h, 4, 2, w, amp)  # warm-up (builds, first launches)

    def timed(grad):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = pic.pic_window(h, K, ck, w, amp, grad=grad)
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    (J, _, _), t_fwd = timed(False)
    (J2, dA, dP), t_grad = timed(True)
    # central difference in the amplitude (1 V): differs from the adjoint
    # where particles reach the walls (the loss events' share of the
    # derivative is not in a pathwise adjoint)
    fd = (pic.pic_window(h, K, ck, w, amp + 1.0, grad=False)[0] -
          pic.pic_window(h, K, ck, w, amp - 1.0, grad=False)[0]) / 2.0
    line = {"metric": "adjoint window: ms per J and per J with gradient", "unit": "ms",
            "value": 1e3 * t_grad, "higher_is_better": False,
            "dtype": "f32 forward + f64 adjoint" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": "c5 adjoint window: R 10 cm, L 2 cm, 65x257 nodes, "
                                   f"{n // 2} e- + {n // 2} Ar+ loaded at n0 1e15 m^-3, collisionless, "
                                   f"{K} steps, checkpoints every {ck}, 100 V at 13.56 MHz; J = time average "
                                   "of the integral of w n_i, w Gaussian at r 3 cm z 1 cm sigma 5 mm",
                       "precision": args.precision},
            "forward_ms": 1e3 * t_fwd, "gradient_ms": 1e3 * t_grad,
            "forward_particle_steps_per_s": n * K / t_fwd,
            "gradient_over_forward": t_grad / t_fwd,
            "J": J, "dJ_damp": dA, "dJ_dphi_zL_max": float(np.abs(dP).max()),
            "dJ_damp_central_difference_1V": fd,
            "particles_lost_in_window": "yes (loaded plasma: electrons reach the walls)"}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--solve-only", action="store_true",
                    help="time only the stand-alone field solve on the workload's mesh")
    ap.add_argument("--particles", type=int, default=0,
                    help="particles per species (default: the workload's; smaller for profiling)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the adjoint window (workload c5) instead")
    ap.add_argument("--ion-subcycle", type=int, default=1,
                    help="move the ions every K-th step with K dt (Sec. 2.7); the count of particle-steps "
                         "then holds each moved ion once per K steps")
    ap.add_argument("--batch", type=int, default=0,
                    help="time a batch of this many independent reactors instead (batched sweep)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.solve_only:
        return solve_only(args) if rank == 0 else 0
    if args.adjoint:
        return adjoint_run(args)
    if args.batch > 0:
        return batch_run(args) if rank == 0 else 0

    if args.impl == "reference":
        if rank != 0:
            return 0
        warm = max(args.warmup, 0)
        import workloads as W
        from oracle import Oracle

        cfg = W.scaled(W.config(args.config), args.cpu_sample)
        o = Oracle(cfg)
        o.load()
        o.step(warm)
        n0 = o.count(0) + o.count(1)
        t0 = time.perf_counter()
        o.step(args.steps)
        dt = time.perf_counter() - t0
        n1 = o.count(0) + o.count(1)
        v = 0.5 * (n0 + n1) * args.steps / dt
        sample = (f"{args.config} mesh and load with {args.cpu_sample} particles per species, "
                  f"{args.steps} timed steps after {warm} warm-up steps, single thread")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": warm, "ms_per_step": 1e3 * dt / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOADS.get(args.config, args.config), "sample": sample},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch

    if world > 1:
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, rank, world)
    main_r = res[args.precision]
    # whole job: units all ranks processed / the slowest rank's time
    e = main_r["e2e"]
    ms_max, psteps_sum, e2e_s, e2e_n = whole_job(main_r["ms"], main_r["psteps"], e["seconds"],
                                                 e["psteps"], world)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    value = psteps_sum / (ms_max * 1e-3)
    peak, peak_kind = _peaks()
    tm = main_r["timings"]
    k_ms = tm["particle_e_ms"] + tm["particle_i_ms"]
    k_bytes = BYTES_PER_PARTICLE[args.precision] * main_r["prof_psteps"]
    achieved = k_bytes / (k_ms * 1e-3) / 1e9 if k_ms > 0 else None
    tb = _traffic(args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS.get(args.config, args.config), "precision": args.precision,
                   "particles_per_rank": main_r["n0"],
                   "l2": f"no flush: particle state ({main_r['n0'] * BYTES_PER_PARTICLE[args.precision] // 2 // 1000000} "
                         f"MB) is larger than L2 (129 MB)",
                   "parallelism": f"{world} independent reactor replica(s), one per GPU",
                   **({"ion_subcycle": args.ion_subcycle} if args.ion_subcycle > 1 else {})},
        "roofline": {"bound": "hbm", "kernel": "k_step (fused particle pass, both species)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_particle": BYTES_PER_PARTICLE[args.precision],
                     "traffic": tb * main_r["prof_psteps"] / (2 * args.steps) if tb else None,
                     "kernel_ms_per_step": k_ms / args.steps},
        "phases_ms_per_step": {k[:-3]: v / args.steps for k, v in tm.items() if k.endswith("_ms")},
        "mg_cycles_per_step": main_r["mg_cycles"],
        "gpu_launches": main_r["launches"],
        "clocks": main_r["clocks"],
        # pic_step's status over the warm-up, the timed steps, the phase pass and
        # the end-to-end steps: anything but PIC_OK voids the line
        "status": _status_name(pic_lib(), first_bad(main_r["statuses"])),
    }
    if "fp64" in res and args.precision != "fp64":
        r = res["fp64"]
        t64 = r["timings"]
        k64 = t64["particle_e_ms"] + t64["particle_i_ms"]
        # the FP64 pass is bound by GB300's FP64 pipe: its FP64 arithmetic
        # against the FP64 FMA rate a plain kernel reaches on this GPU
        fma = pic_lib_rate()
        flops = FP64_FLOPS_PER_PARTICLE * r["prof_psteps"] / (k64 * 1e-3) / 1e9 if k64 > 0 else None
        line["fp64"] = {"value": r["psteps"] / (r["ms"] * 1e-3), "unit": UNIT,
                        "ms_per_step": r["ms"] / args.fp64_steps, "steps": args.fp64_steps,
                        "particle_pass_ms_per_step": k64 / args.fp64_steps,
                        "solve_ms_per_step": t64["solve_ms"] / args.fp64_steps,
                        "mg_cycles_per_step": r["mg_cycles"],
                        "roofline": {"bound": "alu", "kernel": "k_step<double> (both species)",
                                     "achieved": flops, "peak": fma, "unit": "GFLOP/s",
                                     "frac": flops / fma if flops and fma else None,
                                     "peak_source": "measured: pic_fp64_fma_rate (FP64 FMA chains)",
                                     "flops_per_particle": FP64_FLOPS_PER_PARTICLE,
                                     "note": "DFMA, DADD and DMUL only; FP64 conversions and compares "
                                             "issue on the same pipe (profiles/k_step_fp64_c2.md)"}}
    e = main_r["e2e"]
    line["e2e"] = {"value": e2e_n / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": e["h2d"], "d2h_bytes_per_step": e["d2h"],
                   "steps": e["steps"]}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.config, args.cpu_sample, args.cpu_steps)
        line["accuracy_vs_fp64_oracle"] = accuracy_vs_oracle(args.config, args.cpu_sample,
                                                             torch.cuda.current_stream())
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    bad = [first_bad(r["statuses"]) for r in res.values()]
    if any(b != 0 for b in bad):
        print(f"bench: a timed call returned {line['status']} (fp64 leg: "
              f"{_status_name(pic_lib(), bad[-1])}); the figures above are void", file=sys.stderr)
        return 1
    return 0


def pic_lib_rate():
    """The GPU's FP64 FMA rate in GFLOP/s (pic_fp64_fma_rate)."""
    from paper_1001_2969_gb300 import pic

    return pic.pic_fp64_fma_rate(16384)


def first_bad(statuses):
    """The first status other than PIC_OK (0), else 0."""
    return next((int(s) for s in statuses if int(s) != 0), 0)


def pic_lib():
    from paper_1001_2969_gb300 import pic

    return pic.lib()


def _status_name(L, st):
    return L.pic_status_string(int(st)).decode()


if __name__ == "__main__":
    sys.exit(main())
