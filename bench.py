"""Benchmark: cell-updates/s of the adaptive non-hydrostatic step, including the
elliptic solve, at a measured error against the FP64 oracle.

Default workload: the ensemble of 32 uneven 2D landslide runs (grids of
256^2 to 1024^2 cells, 1.58e7 cells in all; plane slopes, elliptic Gaussian
slides moving as s0 ln cosh(t/t0), parameters drawn per member), adaptive
|eta/d| > 1e-3 with the Moore enlargement, FP32 state with the FP64
multigrid-preconditioned solve.  One "step" is one time step of every
member: bottom, two Heun stages, criterion and mask, compaction, assembly,
Krylov solve on the active cells, correction.  The state is advanced
(untimed) --spin-steps steps from still water at t = 0.3 s, then --warmup
steps, then --steps timed steps bracketed by a barrier and stream
synchronisation and timed with CUDA events on the handle's stream (the
state, 4 fields per cell, exceeds the 129 MB L2, so no flush is needed).
--workload slide_1d runs the 1D slide batch (64 members x 50 000 cells).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own ensemble (weak scaling, no collective
on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s incl. NH solve at fixed error vs FP64 oracle; adaptive/learned vs global plain"
UNIT = "cell-updates/s"
WORKLOAD = "1D moving-bottom slide, 64 members x 50000 cells, adaptive |eta/d|>1e-3 + 1-cell enlargement"

# Algorithmic bytes per unit for each kernel class, FP64 path.  Units: cells
# of the whole batch for the predictor, active cells for the rest.
BYTES_PER_UNIT_FP64 = {
    "predict": 56.125,    # read zeta, hu, hw, d0 (32); write zeta~, hu~, hw~ (24); mark bit (1/8)
    "compact": 4.25,      # read mark bits, write dilated bits (2/8) and the int32 list entry
    "assemble": 116.0,    # read zeta~, hu~, hw~, d0, list (36); write 8 coefficients + 2 neighbours (80)
    "solve_init": 84.0,   # read R, 3 coeffs, 2 nbrs, list (44); write x, r, rh, 4 zeroed vectors (..)
    "precond": 88.0,      # fused PCG update + PCR: read 3 coeffs, 2 nbrs, x, p, r_old, q (64); write x, r_new, z (24)
    "pcg_a": 64.0,        # read z, p_old, 3 coeffs, 2 nbrs (48); write p, q (16)
    "pcg_loop": 152.0,    # per PCG iteration: phase A (pcg_a, 64) + phase B (update + PCR, 88)
    "cg_a": 64.0,
    "cg_b": 48.0,
    "correct": 92.0,      # read list, nbrs, x, 4 coeffs, hu, hw (68); write hu, hw, psi (24)
}
# Mixed path: FP32 state and Krylov vectors; FP64 operator, rhs and iterate.
BYTES_PER_UNIT_MIXED = {
    "predict": 28.125,    # read zeta, hu, hw, d0 (16); write 3 fields (12); mark bit
    "compact": 4.25,
    "assemble": 120.0,    # read 3 fields, d0 (FP64), list (24); FP64 op + rhs (32), FP32 op (12), 4 coeffs (16), nbrs (8)
    "solve_init": 44.0,   # k_ir_resid: read R, 3 FP64 coeffs, nbrs, x64 (48, cached neighbours); write rhs32
    "precond": 48.0,      # read 3 FP32 coeffs, 2 nbrs, x, p, r_old, q (36); write x, r_new, z (12)
    "pcg_a": 36.0,
    "pcg_loop": 84.0,     # per inner PCG iteration: 36 + 48
    "correct": 50.0,
}
# The 1D FP64 predictor is bound by the FP64 pipe, not by HBM: its roofline is
# FLOP/s against the FP64 peak.  FP64 FLOPs per cell and step counted from the
# algorithm (each face once, no halo recompute, central slopes): per Heun
# stage the primitives 4, one face 62 (slopes 12, reconstruction 12, depths
# and discharges 6, wave speeds 9, four flux components 23), the cell update
# 17 and the stage 7 to 9: 90 per stage.
FLOPS_PER_CELL_FP64_PREDICT = 180.0
# FP64 peak derived from the unit counts and clock: 152 SMs x 2 DFMA/clk x
# 2 FLOP x 2.07 GHz (the nominal 1.25 TFLOP/s).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


# FP32 state with an FP64 solve: FP32 predictor and correction state, FP64
# operator and Krylov vectors.
BYTES_PER_UNIT_MIXED64 = {
    "predict": 28.125,
    "compact": 4.25,
    "assemble": 80.0,     # read 3 FP32 fields, FP64 d0, list (24); write FP64 op + rhs (32), 4 FP32 coeffs (16), nbrs (8)
    "solve_init": 84.0,
    "precond": 88.0,
    "pcg_a": 64.0,
    "pcg_loop": 152.0,
    "correct": 60.0,      # read list, nbrs, x (FP64), 4 FP32 coeffs, hu, hw; write hu, hw, psi
}


def _load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed0(members, rank):
    """Seed offset of a rank's batch: rank r draws members r*M .. r*M + M - 1,
    so every rank runs its own independent members (weak scaling)."""
    return members * rank


def max_over_ranks(x, ws, device):
    """The slowest rank's time (all ranks get it); x itself when ws == 1."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _oracle_sample(wl, max_steps, budget_s, crit):
    """Oracle (FP64 C, one host thread) on member 0 from t = 0: cell-updates/s."""
    import oracle as O
    m = wl.members[0]
    p = O.Params(nx=m.nx, dx=m.dx, xl=m.xl, slide=m.slide, A=m.A, L=m.L, xc0=m.xc0, s0=m.s0,
                 t0=m.t0, crit=crit, knh=1e-3, enlarge=1, rtol=1e-12, max_iter=20000)
    s = O.State(m.h, m.hu, m.hw)
    t0 = time.perf_counter()
    k = 0
    while k < max_steps and time.perf_counter() - t0 < budget_s:
        O.step(p, m.d0, k * wl.dt, k, wl.dt, s)
        k += 1
    el = time.perf_counter() - t0
    return m.nx * k / el, k, el


def run_reference(args):
    """The oracle arm: each step is one time step of one 50 000-cell member."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2505_17025_gb300 import workloads as W
    import oracle as O
    wl = W.slide_1d(n_members=1)
    m = wl.members[0]
    p = O.Params(nx=m.nx, dx=m.dx, xl=m.xl, slide=m.slide, A=m.A, L=m.L, xc0=m.xc0, s0=m.s0,
                 t0=m.t0, crit=O.CRIT_ETA_D, knh=1e-3, enlarge=1, rtol=1e-12, max_iter=20000)
    s = O.State(m.h, m.hu, m.hw)
    for k in range(args.warmup):
        O.step(p, m.d0, k * wl.dt, k, wl.dt, s)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        O.step(p, m.d0, k * wl.dt, k, wl.dt, s)
    el = time.perf_counter() - t0
    v = m.nx * args.steps / el
    sample = (f"member 0 of the 64-member batch (50000 cells), time steps {args.warmup}.."
              f"{args.warmup + args.steps - 1} from t = 0, FP64 C oracle, 1 thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle: one member per step)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def compare_forms(wl, G0, t_now, args):
    """Wall time per step of the method's forms on the same batch, each started
    from G0's state at t_now: global FP64 with the plain warm start (every cell
    non-hydrostatic), adaptive FP64, and adaptive FP64 / mixed precision with
    the learned start (network trained on pairs harvested from the first
    steps, outside the timed region)."""
    import torch
    from paper_2505_17025_gb300 import guess_train as GT
    from paper_2505_17025_gb300 import nhswe as N
    h, hu, hw, _ = G0.get_state()
    forms = [("global_fp64_plain", N.NH_FP64, N.NH_CRIT_GLOBAL, False),
             ("adaptive_fp64", N.NH_FP64, N.NH_CRIT_ETA_D, False),
             ("adaptive_fp64_learned", N.NH_FP64, N.NH_CRIT_ETA_D, True),
             ("adaptive_mixed_learned", N.NH_MIXED, N.NH_CRIT_ETA_D, True),
             ("adaptive_fp32state_fp64solve", N.NH_MIXED_FP64_SOLVE, N.NH_CRIT_ETA_D, False),
             ("adaptive_fp32state_fp64solve_learned", N.NH_MIXED_FP64_SOLVE, N.NH_CRIT_ETA_D, True)]
    k_steps = max(1, args.form_steps)
    cells = sum(m.nx for m in wl.members)
    out = {}
    for name, prec, crit, learned in forms:
        G = N.grid_from_workload(wl, precision=prec)
        G.set_state(h, hu, hw, t_now)
        G.set_criterion(crit, 1e-3, 1, False)
        rtol = 1e-10 if prec == N.NH_MIXED else 1e-12
        G.set_solver(N.NH_SOLVER_AUTO, rtol, 20000, N.NH_GUESS_PREV)
        t_train = 0.0
        if learned:
            G.cnn_attach()
            t0 = time.perf_counter()
            samples = GT.collect(G, wl.dt, args.form_harvest)
            G.cnn_record(False)
            if samples:
                params, _ = GT.train(samples, steps=args.form_train)
                G.cnn_set_params(params)
            G.set_solver(N.NH_SOLVER_AUTO, rtol, 20000, N.NH_GUESS_CNN)
            t_train = time.perf_counter() - t0
        G.run(wl.dt, max(3, args.warmup))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(G.stream)
        st, info = G.run(wl.dt, k_steps)
        e1.record(G.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k_steps
        rec = {"ms_per_step": ms, "cell_updates_per_s": cells / (ms * 1e-3),
               "krylov_iters_per_step": info["iters_total"] / k_steps,
               "active_cells_per_step": info["active_total"] / k_steps,
               "error_bound_vs_oracle": "1e-9 a" if prec == N.NH_FP64 else "1e-4 a (while masks agree)",
               "precision": {N.NH_FP64: "fp64", N.NH_MIXED: "fp32 state + fp32 krylov in fp64 refinement",
                             N.NH_MIXED_FP64_SOLVE: "fp32 state + fp64 krylov"}[prec]}
        if learned:
            rec["starts"] = G.cnn_choices()
            rec["harvest_and_train_s"] = t_train
        out[name] = rec
        G.close()
    base = out["global_fp64_plain"]["ms_per_step"]
    return {"steps": k_steps, "t_start": t_now, "forms": out,
            "speedup_vs_global_fp64_plain": {k: base / v["ms_per_step"] for k, v in out.items()}}


def time_network(wl, args):
    """The learned-guess network's fused forward (tcgen05, BF16 x BF16 -> FP32)
    on the whole batch (every cell a network input), CUDA events over 20
    launches after 3 warm-up launches; FLOPs = 2 x 9216 multiply-adds per
    cell (the four layers' 3 c_in c_out), tile halos not counted."""
    import torch
    from paper_2505_17025_gb300 import guess_train as GT
    from paper_2505_17025_gb300 import nhswe as N
    nb = len(wl.members)
    pitch = (max(m.nx for m in wl.members) + 511) // 512 * 512
    g = torch.Generator(device="cuda").manual_seed(0)
    feat = torch.randn((nb, pitch, N.NH_CNN_IN), generator=g, device="cuda").to(torch.bfloat16)
    nxd = torch.tensor([m.nx for m in wl.members], dtype=torch.int32, device="cuda")
    params = GT.init_params(0, last_gain=1.0)
    y = torch.zeros((nb, pitch), dtype=torch.float32, device="cuda")
    import ctypes as C
    L = N.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args_c = (C.c_void_p(feat.data_ptr()), C.c_void_p(nxd.data_ptr()), nb, pitch, C.c_void_p(params.data_ptr()),
              C.c_void_p(y.data_ptr()), 1.0, None, stream)

    def fwd():
        rc = L.nh_cnn_forward(*args_c)
        if rc != 0:
            raise RuntimeError(f"nh_cnn_forward: {rc}")

    for _ in range(3):
        fwd()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 20
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fwd()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    cells = sum(m.nx for m in wl.members)
    flops = 2.0 * 9216 * cells
    peaks, kind = _load_peaks()
    tf = flops / (ms * 1e-3) / 1e12
    return {"kernel": "k_forward", "cells": cells, "ms_per_launch": ms, "tflops": tf,
            "bf16_peak_tflops": peaks.get("bf16_tflops"), "frac": tf / peaks.get("bf16_tflops", 1900.0),
            "launch": "C ABI nh_cnn_forward on preallocated buffers, back to back on one stream"}


def _landslide_h(wl, t):
    """Still water over the slide's position at time t."""
    sl = wl.slide
    s = sl["s0"] * math.log(math.cosh(t / sl["t0"]))
    x = (np.arange(wl.nx) + 0.5) * wl.dx
    y = (np.arange(wl.ny) + 0.5) * wl.dy
    X, Y = np.meshgrid(x, y)
    return wl.d0 - sl["A"] * np.exp(-((X - sl["xc0"] - s) / sl["Lx"]) ** 2 - ((Y - sl["yc0"]) / sl["Ly"]) ** 2)


def _workload_2d(args):
    """(members, dt, description, k_nh, t_start) of a 2D workload."""
    from paper_2505_17025_gb300 import workloads as W
    knh = args.knh or 1e-3
    if args.workload == "line_soliton_2d":
        w = W.line_soliton_2d()
        return [w], w.dt, f"line_soliton_2d {w.nx}x{w.ny}, dx {w.dx} m, periodic, a/h 0.2", knh, 0.0
    if args.workload == "landslide_2d":
        w = W.landslide_2d()
        return [w], w.dt, f"landslide_2d {w.nx}x{w.ny}, dx {w.dx} m, slope 0.2, walls", knh, 0.3
    _, rank, _ = _dist()
    wls, dt = W.landslide_ensemble_2d(n_members=args.ens_members, seed0=rank_seed0(args.ens_members, rank))
    return (wls, dt, f"landslide_ensemble_2d: {len(wls)} runs, nx, ny drawn from 256..1024 (step 64), dx 0.02 m, "
            f"tan(theta) U(0.1,0.3), A U(0.05,0.15), Lx U(0.5,1.5), s0 U(1,3); member m seeded with m "
            f"(+ {args.ens_members} x rank)",
            knh, 0.3)


def _initial_2d(w, t_start):
    """Member's state at t_start: the workload's own, or still water over the slide."""
    return (_landslide_h(w, t_start) if w.slide else w.h), w.hu, w.hv, w.hw


def _save_member(path, w, fields):
    sl = w.slide or {}
    np.savez(path, h=fields[0], hu=fields[1], hv=fields[2], hw=fields[3], d0=w.d0,
             geo=np.array([w.nx, w.ny, w.bc_x, w.bc_y], dtype=np.int64), sp=np.array([w.dx, w.dy]),
             slide=np.array([1.0 if w.slide else 0.0] + [float(sl.get(k, 0.0)) for k in
                                                         ("A", "Lx", "Ly", "xc0", "yc0", "s0", "t0")]),
             amp=np.array([w.amplitude]))


def _oracle2d_job(job):
    """Worker (a spawned process): the FP64 2D oracle on one member from a
    handed-over state saved by _save_member.  job = (path, crit, k_nh, t0,
    step0, dt, n_steps, checkpoints); returns (path, {step: (h, hu, hv, hw,
    mask)}, seconds, cells x steps, iterations)."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    import oracle.oracle2d as O2
    path, crit, knh, t0, step0, dt, n, checks = job[:8]
    write_back = len(job) > 8 and job[8]
    z = np.load(path)
    nx, ny, bcx, bcy = (int(v) for v in z["geo"])
    p = O2.Params2D(nx=nx, ny=ny, dx=float(z["sp"][0]), dy=float(z["sp"][1]), bcx=bcx, bcy=bcy, crit=crit,
                    knh=knh, enlarge=1, rtol=1e-13)
    sl = z["slide"]
    if sl[0] > 0:
        p.slide = O.SLIDE_GAUSS_LNCOSH
        p.A, p.Lx, p.Ly, p.xc0, p.yc0, p.s0, p.t0 = (float(v) for v in sl[1:])
    d0 = z["d0"]
    s = O2.State2D(z["h"], z["hu"], z["hv"], z["hw"], z["q"] if "q" in z.files else None)
    out, iters = {}, 0
    t_begin = time.perf_counter()
    for k in range(n):
        st, info, mk = O2.step(p, d0, t0 + k * dt, step0 + k, dt, s, want_mask=True)
        if st != O.OK:
            raise RuntimeError(f"oracle {path} step {k}: status {st}")
        iters += info["iters"]
        if k + 1 in checks:
            out[k + 1] = tuple(a.reshape(ny, nx).copy() for a in (s.h, s.hu, s.hv, s.hw)) + (mk.copy(),)
    el = time.perf_counter() - t_begin
    if write_back:
        np.savez(path, h=s.h, hu=s.hu, hv=s.hv, hw=s.hw, q=s.q, d0=d0, geo=z["geo"], sp=z["sp"], slide=z["slide"],
                 amp=z["amp"])
    return path, out, el, nx * ny * n, iters


def _pool(n):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(processes=n)


def _ncores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _errors_2d(w, got, ref):
    """max |d eta| / a and the momenta / (a sqrt(g h_max)) between two
    (h, hu, hv, hw[, mask]) tuples of one member, and the mask cells that differ."""
    a = w.amplitude
    qs = a * math.sqrt(9.81 * float(np.max(w.d0)))
    e = [float(np.max(np.abs(got[0] - ref[0]))) / a]
    e += [float(np.max(np.abs(got[q] - ref[q]))) / qs for q in (1, 2, 3)]
    return e


def _grid_2d(N, wls, precision, crit, knh, precond, t, states, rtol=1e-12):
    G = N.Grid2D.ensemble([dict(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, d0=w.d0, bc_x=w.bc_x, bc_y=w.bc_y)
                           for w in wls])
    if precision == "mixed64":
        G.set_precision(N.NH_MIXED_FP64_SOLVE)
    for i, w in enumerate(wls):
        if w.slide:
            G.set_bottom_motion(w.slide, member=i)
        G.set_state(*states[i][:4], t=t, member=i)
    G.set_criterion(crit, knh, 1)
    G.set_solver(rtol, 20000, N.NH_GUESS_PREV)
    G.set_preconditioner(precond)
    return G


# Algorithmic bytes of the 2D kernel classes.  Predictor: the fused minimum
# of a Heun step is to read Q^n and write Q~ once (4 fields each: 64 B per
# cell in FP64, 32 B with FP32 state); the FP64 state's two stage launches
# share it (one launch is credited half), the FP32 state's one-launch
# predictor is credited all of it.  Krylov solve: per active cell and
# iteration the fused CG minimum, 24 B in FP32, 48 B with FP64 vectors.  The
# bottom is in-register work in the minimum (0 B).
BYTES_2D_STAGE = {"fp64": 32.0, "mixed64": 32.0}
# Tile candidates of the one-launch FP32 predictor (nh2d_set_tile).
PRED_TILES = ("32x16", "64x8", "32x8", "64x16")
SOLVE_BYTES_PER_ITER = 48.0
# Solve tolerance of the FP32-state form (relative residual).  Its error
# against the oracle is set by the FP32 state (eta carries about 1e-7 m of
# rounding): on the ensemble's timed window 1e-12, 1e-10 and 1e-9 all give
# max |d eta| = 1.7e-7 to 1.8e-7 a (40, 34 and 30 iterations per step); at
# 1e-8 the solve's own error shows (3.5e-6 a).  The FP64 forms keep 1e-12.
RTOL_FP32_STATE = 1e-9
# FP64 FLOPs per cell of one stage, counted from the algorithm (central
# slopes, each face once, no halo recompute): primitives 5, two faces of 82
# (slopes 16, reconstruction 18, depths and discharges 6, wave speeds 9,
# five flux components 33), cell update 55 (slopes and face thicknesses 18,
# four rates 32, the stage 5 to 10).
FLOPS_2D_STAGE_FP64 = 229.0


def run_2d(args):
    """The 2D workloads: --workload landslide_ensemble_2d (default; 32
    uneven landslide runs of 256^2 to 1024^2 cells), landslide_2d (2048^2)
    or line_soliton_2d (1024^2, periodic).  The state is advanced --spin-steps
    untimed steps from t_start (still water over the slide at t = 0.3 s) so
    the timed window sees a developed wave field, then --warmup steps, then
    --steps timed steps replayed from the captured graph (CUDA events on the
    handle's stream, nvidia-smi clocks sampled meanwhile).  Around the window:
    the error against the FP64 oracle run from the same hand-off on sampled
    members; a second, event-profiled pass for per-kernel times and the
    roofline; an end-to-end pass through the C ABI with pinned host buffers;
    the method's forms from the window's start (global FP64, adaptive FP64,
    adaptive FP32 state, the line-preconditioned solve) with their own errors;
    and the oracle timed on one host thread and on all host cores."""
    import torch
    from paper_2505_17025_gb300 import nhswe as N
    import oracle as O
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wls, dt, name, knh, t_start = _workload_2d(args)
    crit = N.NH_CRIT_GLOBAL if args.mode == "global" else N.NH_CRIT_ETA_D
    ocrit = O.CRIT_GLOBAL if args.mode == "global" else O.CRIT_ETA_D
    precond = N.NH_PRECOND_LINE if args.precond == "line" else N.NH_PRECOND_MG
    if args.precision == "mixed":
        raise SystemExit("2D grids: --precision fp64 or mixed64 (FP32 state, FP64 solve)")
    init = [_initial_2d(w, t_start) for w in wls]
    G = _grid_2d(N, wls, args.precision, crit, knh, precond, t_start, init, rtol=args.rtol)
    cells = sum(w.nx * w.ny for w in wls)
    t_spin0 = time.perf_counter()
    if args.spin_steps:
        G.run(dt, args.spin_steps)
    torch.cuda.synchronize()
    t_spin = time.perf_counter() - t_spin0
    warm = max(3, args.warmup)
    G.run(dt, warm)
    n_before = args.spin_steps + warm
    t0 = t_start + n_before * dt
    # hand-off at the window's start: every member's FP64 state
    handoff = [tuple(G.get_state(i)[:4]) for i in range(len(wls))]
    order = sorted(range(len(wls)), key=lambda i: wls[i].nx * wls[i].ny)
    sample = order[:max(1, min(args.err_members, len(wls)))]
    tmpdir = tempfile.mkdtemp(prefix="nhbench")
    paths = {}
    for i in range(len(wls)):
        paths[i] = os.path.join(tmpdir, f"m{i}.npz")
        _save_member(paths[i], wls[i], handoff[i])

    # ---- timed window
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.profiler.start()
    e0.record(G.stream)
    st, info = G.run(dt, args.steps)
    e1.record(G.stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    graph_runs = G.graph_runs
    tile = G.set_tile(-1)
    final = {i: tuple(G.get_state(i)[:4]) + (G.get_mask(i),) for i in sample}
    value = ws * cells * args.steps / (ms * 1e-3)

    # ---- the oracle from the same hand-off (sampled members), in worker processes
    n_form = max(1, args.form_steps)
    checks = sorted({args.steps, n_form})
    jobs = [(paths[i], ocrit, knh, t0, n_before, dt, max(checks), set(checks)) for i in sample]
    pool = _pool(min(len(jobs) + 1, _ncores()))
    err_async = pool.map_async(_oracle2d_job, jobs)
    jobs_g = [(paths[sample[0]], O.CRIT_GLOBAL, knh, t0, n_before, dt, n_form, {n_form})] if args.form_steps else []
    err_g_async = pool.map_async(_oracle2d_job, jobs_g) if jobs_g else None

    # ---- profiled pass: per-kernel device times (events on the handle's stream)
    G.set_profiling(True)
    st2, info2 = G.run(dt, args.steps)
    prof = G.get_profile()
    G.set_profiling(False)
    iters_prof = info2["iters_total"] / max(1, args.steps)
    act_prof = info2["active_total"] / max(1, args.steps)

    # ---- end to end through the C ABI: pinned host state in, step, state out
    e2e = None
    if args.e2e_steps > 0:
        hb = [[torch.empty(w.nx * w.ny, dtype=torch.float64, pin_memory=True) for _ in range(4)] for w in wls]
        for i in range(len(wls)):
            G.get_state_ptr(i, *(b.data_ptr() for b in hb[i]))
        torch.cuda.synchronize()
        tt0 = time.perf_counter()
        for k in range(args.e2e_steps):
            for i in range(len(wls)):
                G.put_state_ptr(i, *(b.data_ptr() for b in hb[i]))
            G.run(dt, 1)
            for i in range(len(wls)):
                G.get_state_ptr(i, *(b.data_ptr() for b in hb[i]))
        el = time.perf_counter() - tt0
        nbytes = 4 * 8 * cells
        e2e = {"value": ws * cells * args.e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps,
               "path": "nh2d_put_member_state (pinned host, all members) + nh2d_run(1) + nh2d_get_member_state"}
    G.close()

    # ---- the method's forms from the window's start (timed on the device)
    forms = {}
    if args.form_steps > 0:
        flist = [("adaptive_fp64_mg", "fp64", crit, N.NH_PRECOND_MG),
                 ("adaptive_fp32state_mg", "mixed64", crit, N.NH_PRECOND_MG),
                 ("adaptive_fp64_line", "fp64", crit, N.NH_PRECOND_LINE),
                 ("global_fp64_mg", "fp64", N.NH_CRIT_GLOBAL, N.NH_PRECOND_MG)]
        for fname, prec, fcrit, fpc in flist:
            F = _grid_2d(N, wls, prec, fcrit, knh, fpc, t0, handoff,
                         rtol=RTOL_FP32_STATE if prec == "mixed64" else 1e-12)
            fe0 = torch.cuda.Event(enable_timing=True)
            fe1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            fe0.record(F.stream)
            _, finfo = F.run(dt, n_form)
            fe1.record(F.stream)
            torch.cuda.synchronize()
            fms = fe0.elapsed_time(fe1) / n_form
            forms[fname] = {"ms_per_step": fms, "cell_updates_per_s": cells / (fms * 1e-3),
                            "solve_rtol": RTOL_FP32_STATE if prec == "mixed64" else 1e-12,
                            "krylov_iters_per_step": finfo["iters_total"] / n_form,
                            "active_cells_per_step": finfo["active_total"] / n_form,
                            "precision": "f64" if prec == "fp64" else "f32 state, f64 solve",
                            "preconditioner": "multigrid" if fpc == N.NH_PRECOND_MG else "x-line",
                            "steps": n_form, "first_solve_from_zero": True}
            forms[fname]["_state"] = {i: tuple(F.get_state(i)[:4]) + (F.get_mask(i),) for i in sample}
            F.close()
            del F

    # ---- errors against the oracle
    ref = {}
    for path, out, el, cu, it in err_async.get():
        ref[path] = out
    worst = [0.0] * 4
    mask_diff = 0
    per_member = {}
    for i in sample:
        r = ref[paths[i]][args.steps]
        e = _errors_2d(wls[i], final[i], r)
        d = int(np.sum(final[i][4] != r[4]))
        mask_diff += d
        worst = [max(u, v) for u, v in zip(worst, e)]
        per_member[str(i)] = {"cells": wls[i].nx * wls[i].ny, "max_d_eta_over_a": e[0], "mask_cells_differ": d}
    bound = 1e-9 if args.precision == "fp64" else 1e-4
    error = {"max_d_eta_over_a": worst[0], "max_d_momentum_over_a_sqrt_gh": max(worst[1:]),
             "bound": bound, "meets_bound": max(worst) <= bound, "mask_cells_differ": mask_diff,
             "members": per_member, "steps": args.steps,
             "how": (f"the FP64 2D oracle run from the GPU state handed over at the window's start "
                     f"(t = {t0:.4f} s, step {n_before}) on the {len(sample)} smallest members, "
                     f"the same {args.steps} steps; states compared cell for cell")}
    if forms:
        ref_g = {p: o for p, o, *_ in err_g_async.get()} if err_g_async else {}
        for fname, rec in forms.items():
            fstate = rec.pop("_state")
            glob = fname.startswith("global")
            ew, dm = 0.0, 0
            for i in sample:
                if glob:
                    if i != sample[0]:
                        continue
                    r = ref_g[paths[i]][n_form]
                else:
                    r = ref[paths[i]][n_form]
                e = _errors_2d(wls[i], fstate[i], r)
                ew = max(ew, max(e))
                dm += int(np.sum(fstate[i][4] != r[4]))
            b = 1e-9 if rec["precision"] == "f64" else 1e-4
            rec.update({"max_error_over_a": ew, "bound": b, "meets_bound": ew <= b, "mask_cells_differ": dm})
        base = forms["global_fp64_mg"]["ms_per_step"]
        speed = {k: base / v["ms_per_step"] for k, v in forms.items()}
    pool.close()
    pool.join()

    # ---- roofline of the kernel class with the largest device time
    peaks, peak_kind = _load_peaks()
    mg = precond == N.NH_PRECOND_MG
    name_k, (dms, dn) = max(((k, v) for k, v in prof.items() if v[1] > 0), key=lambda kv: kv[1][0])
    t_launch = dms * 1e-3 / dn
    kernel_name = {"solve": "k2_mg_pcg" if mg else "k_pcg_persistent", "stage": "k2_stage"}.get(name_k,
                                                                                            f"k2_{name_k}")
    if name_k == "stage" and args.precision == "fp64":
        flops = FLOPS_2D_STAGE_FP64 * cells
        ach = flops / t_launch / 1e12
        pk = FP64_PEAK_GFLOPS / 1e3
        roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "traffic": None,
                "kernel": kernel_name, "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (FP64 pipe)",
                "flops_per_launch": flops,
                "hbm_frac": BYTES_2D_STAGE["fp64"] * cells / t_launch / 1e9 / peaks["hbm_gbs"]}
    else:
        if name_k == "stage":
            bpl = BYTES_2D_STAGE[args.precision] * cells
        elif name_k == "solve":
            bpl = SOLVE_BYTES_PER_ITER * act_prof * iters_prof
        else:
            bpl = None
        ach = bpl / t_launch / 1e9 if bpl else None
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"] if ach else None, "traffic": None, "kernel": kernel_name,
                "peak_kind": peak_kind, "bytes_per_launch": bpl}
    roof.update({"launches_per_step": dn / args.steps, "avg_launch_us": 1e6 * t_launch,
                 "share_of_device_time": dms / max(1e-12, sum(v[0] for v in prof.values()))})
    solve_ms = prof["solve"][0]
    solve_info = {"ms_per_step": solve_ms / max(1, args.steps), "krylov_iters_per_step": iters_prof,
                  "active_cells_per_step": act_prof,
                  "bytes_per_active_cell_and_iteration": SOLVE_BYTES_PER_ITER,
                  "achieved_gbs": (SOLVE_BYTES_PER_ITER * act_prof * iters_prof * args.steps
                                   / max(solve_ms * 1e-3, 1e-12) / 1e9)}
    stage_ms, stage_n = prof["stage"]
    stage_info = {"ms_per_launch": stage_ms / max(1, stage_n),
                  "achieved_gbs": BYTES_2D_STAGE[args.precision] * cells / max(stage_ms * 1e-3 / max(1, stage_n),
                                                                               1e-12) / 1e9}

    # ---- the oracle on the host cores, on the same window (hand-off at t0)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = _cpu_baseline_2d(wls, paths, order, ocrit, knh, t0, n_before, dt, args)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": warm, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32 state, f64 solve",
               "data": "synthetic",
               "config": {"workload": name, "cells": cells, "members": len(wls), "mode": args.mode,
                          "precision": args.precision,
                          "preconditioner": "multigrid" if precond == N.NH_PRECOND_MG else "x-line",
                          "predictor_tile": (PRED_TILES[tile] if args.precision == "mixed64" and tile >= 0
                                             else "32x8 two-launch stages (FP64 state)"),
                          "k_nh": knh, "solve_rtol": args.rtol, "t_start": t_start, "spin_up_steps": args.spin_steps,
                          "spin_up_s": t_spin, "window_t0": t0, "dt": dt,
                          "mean_active_cells_per_step": info["active_total"] / max(1, args.steps),
                          "mean_krylov_iters_per_step": info["iters_total"] / max(1, args.steps),
                          "l2": "inputs larger than the 129 MB L2 (state 4 x 8 B x cells); no flush"},
               "error_vs_oracle": error,
               "roofline": roof, "solve": solve_info, "stage": stage_info, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": sum(n for _, n in prof.values()) + (2 * prof["solve"][1] if mg else 0),
               "timed_region": f"nh2d_run replaying the captured step graph ({graph_runs} graph run(s))",
               "clocks": clk,
               "kernel_ms": {k: v[0] for k, v in prof.items() if v[1] > 0},
               "kernel_launches": {k: v[1] for k, v in prof.items() if v[1] > 0}}
        if forms:
            out["forms"] = {"t0": t0, "forms": forms, "speedup_vs_global_fp64_mg": speed,
                            "note": "each form from the FP64 state at the window's start; first solve from "
                                    "a zero guess; errors against the oracle over the same steps"}
        print(json.dumps(out))
    shutil.rmtree(tmpdir, ignore_errors=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _cpu_baseline_2d(wls, paths, order, ocrit, knh, t0, step0, dt, args):
    """The oracle as it stands on the window's hand-off: one host thread on
    the smallest member, and every member at once on all host cores (one
    process per member, up to the core count)."""
    one = _oracle2d_job((paths[order[0]], ocrit, knh, t0, step0, dt, args.cpu_steps, set()))
    v1 = one[3] / one[2]
    nc = _ncores()
    pool = _pool(min(nc, len(wls)))
    t_begin = time.perf_counter()
    res = pool.map(_oracle2d_job, [(paths[i], ocrit, knh, t0, step0, dt, 1, set()) for i in range(len(wls))])
    el = time.perf_counter() - t_begin
    pool.close()
    pool.join()
    cu = sum(r[3] for r in res)
    return {"value": cu / el, "unit": UNIT, "cores": min(nc, len(wls)), "kind": "oracle",
            "one_thread": {"value": v1, "cores": 1,
                           "sample": f"member {order[0]} ({wls[order[0]].nx}x{wls[order[0]].ny}), "
                                     f"{args.cpu_steps} steps from the window's start"},
            "sample": (f"all {len(wls)} members, one time step from the window's hand-off (t = {t0:.4f} s), "
                       f"one spawned process per member on {min(nc, len(wls))} of {nc} host cores; "
                       f"FP64 C oracle as it stands")}


def run_reference_2d(args):
    """The oracle arm on the 2D workload: every member from the workload's own
    start (t = 0.3 s, still water over each slide; the GPU arm's spin-up is
    out of reach of the oracle in minutes), one process per member on the
    host cores; --warmup untimed steps, then --steps timed steps (one step =
    one time step of every member)."""
    import oracle as O
    ws, rank, _ = _dist()
    if rank != 0:
        return
    wls, dt, name, knh, t_start = _workload_2d(args)
    ocrit = O.CRIT_GLOBAL if args.mode == "global" else O.CRIT_ETA_D
    tmpdir = tempfile.mkdtemp(prefix="nhref")
    paths = []
    for i, w in enumerate(wls):
        paths.append(os.path.join(tmpdir, f"m{i}.npz"))
        _save_member(paths[-1], w, _initial_2d(w, t_start))
    nc = _ncores()
    pool = _pool(min(nc, len(wls)))
    if args.warmup:
        pool.map(_oracle2d_job, [(p, ocrit, knh, t_start, 0, dt, args.warmup, set(), True) for p in paths])
    t1 = t_start + args.warmup * dt
    tb = time.perf_counter()
    res = pool.map(_oracle2d_job, [(p, ocrit, knh, t1, args.warmup, dt, args.steps, set(), True) for p in paths])
    el = time.perf_counter() - tb
    pool.close()
    pool.join()
    shutil.rmtree(tmpdir, ignore_errors=True)
    cells = sum(w.nx * w.ny for w in wls)
    v = cells * args.steps / el
    sample = (f"all {len(wls)} members, steps {args.warmup}..{args.warmup + args.steps - 1} from t = {t_start} s "
              f"(still water over each slide), one spawned process per member on {min(nc, len(wls))} of {nc} "
              f"host cores, FP64 C oracle as it stands")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name + " (oracle)", "cells": cells, "members": len(wls), "k_nh": knh,
                   "t_start": t_start},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": min(nc, len(wls)), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def _ratio_cases():
    """The paper's 1D cases with their own dx, dt and duration: the solitary
    wave of Sec. 4.1 (a = 2 m, d = 10 m, 800 m, 200 cells, dt 0.1 s, 30 s),
    the plate moved up and down (Sec. 4.2) and the sliding block at the three
    Froude numbers (Sec. 4.3)."""
    from paper_2505_17025_gb300 import workloads as W
    sol = W.solitary_1d(nx=200, length=800.0, depth=10.0, a=2.0, T=30.0)
    cases = [("solitary", sol, 0.1, 300), ("plate_up", W.plate_1d(up=True), None, None),
             ("plate_down", W.plate_1d(up=False), None, None)]
    for r, fr in enumerate(("0.125", "0.25", "0.375")):
        cases.append((f"block_fr{fr}", W.block_1d(row=r), None, None))
    return cases


def run_paper_ratios(args):
    """GPU wall time of the adaptive runs relative to the global run
    (t_local / t_global) for the six criteria of Sec. 5.1, plain and enlarged
    by one cell (Sec. 5.2), on the paper's 1D cases, beside the paper's
    printed ratios.  Each run: the whole simulation from t = 0, replayed from
    captured graphs, timed with CUDA events after one untimed capture run;
    one member alone (latency-bound: about 1 000 cells), and a batch of
    --members copies of it in one handle (the GPU loaded)."""
    import copy
    import torch
    from paper_2505_17025_gb300 import nhswe as N
    with open(os.path.join(ROOT, "tests", "golden", "paper_time_ratios.json")) as f:
        paper = json.load(f)
    crits = [("eta_d", N.NH_CRIT_ETA_D), ("eta_x", N.NH_CRIT_ETA_X), ("u", N.NH_CRIT_U),
             ("u_x", N.NH_CRIT_U_X), ("w", N.NH_CRIT_W), ("w_x", N.NH_CRIT_W_X)]
    out = {}
    for name, wl, dt, n in _ratio_cases():
        dt = dt or wl.dt
        n = n or wl.n_steps
        m0 = wl.members[0]
        res = {}
        for batch in (1, args.members):
            wlb = copy.copy(wl)
            wlb.members = [m0] * batch

            def timed(crit, enlarge, first):
                G = N.grid_from_workload(wlb)
                G.set_criterion(crit, 1e-3, enlarge, first)
                G.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000, N.NH_GUESS_PREV)
                G.run(dt, 3)
                G.set_state([m0.h] * batch, [m0.hu] * batch, [m0.hw] * batch, 0.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(G.stream)
                st, info = G.run(dt, n)
                e1.record(G.stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                share = info["active_total"] / float(m0.nx * batch * n)
                G.close()
                return ms, share

            tg, _ = timed(N.NH_CRIT_GLOBAL, 1, False)
            rec = {"global_ms": tg}
            for key, enl in (("plain", 0), ("enlarged", 1)):
                rows = {}
                for ci, (cn, ck) in enumerate(crits):
                    t, share = timed(ck, enl, cn in ("w", "w_x"))
                    rows[cn] = {"gpu": t / tg, "active_share": share, "paper": paper[key][name][ci]}
                rec[key] = rows
            res[f"batch_{batch}"] = rec
        out[name] = {"cells": m0.nx, "steps": n, "dt": dt, "runs": res}
    print(json.dumps({"paper_time_ratios": out, "k_nh": 1e-3,
                      "note": "t_local / t_global of whole runs on one GB300; the paper's ratios are "
                              "from its own DG implementation on unstated hardware (context only)"}))


def run_ours(args):
    import torch
    from paper_2505_17025_gb300 import nhswe as N
    from paper_2505_17025_gb300 import workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    wl = W.slide_1d(n_members=args.members, seed0=rank_seed0(args.members, rank))
    prec = {"fp64": N.NH_FP64, "mixed": N.NH_MIXED, "mixed64": N.NH_MIXED_FP64_SOLVE}[args.precision]
    G = N.grid_from_workload(wl, precision=prec)
    crit = N.NH_CRIT_GLOBAL if args.mode == "global" else N.NH_CRIT_ETA_D
    G.set_criterion(crit, 1e-3, 1, False)
    rtol = 1e-10 if args.precision == "mixed" else 1e-12
    G.set_solver(N.NH_SOLVER_AUTO, rtol, 20000, N.NH_GUESS_PREV)
    G.set_preconditioner(N.NH_PRECOND_LINE if args.precond == "line" else N.NH_PRECOND_NONE)
    cells = wl.members[0].nx * len(wl.members)

    n_spin = int(round(args.t_start / wl.dt))
    t_spin0 = time.perf_counter()
    if n_spin:
        G.run(wl.dt, n_spin)
    t_spin = time.perf_counter() - t_spin0
    G.run(wl.dt, args.warmup)

    stream = G.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    G.set_profiling(False)
    clocks.start()
    # profiler range = the timed steps (an ncu run with --profile-from-start off
    # records exactly these launches; no effect otherwise)
    torch.cuda.profiler.start()
    e0.record(stream)
    st, info = G.run(wl.dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    # second pass of the same length, step by step with every kernel bracketed by
    # CUDA events on the library's stream: per-kernel device times for the roofline
    G.set_profiling(True)
    st2, info2 = G.run(wl.dt, args.steps)
    prof = G.get_profile()
    G.set_profiling(False)
    launches_profiled = sum(n for _, n in prof.values())
    ms = max_over_ranks(ms, ws, "cuda")
    value = ws * cells * args.steps / (ms * 1e-3)
    # kernels per step of the timed (graph-replayed) region: the profiled pass
    # runs the same kernel sequence, so its launch count per step applies
    launches = launches_profiled
    act_mean = info["active_total"] / max(args.steps, 1)
    iters_mean = info["iters_total"] / max(args.steps, 1)

    # dominant kernel class by device time, its algorithmic bytes per launch
    table = {"fp64": BYTES_PER_UNIT_FP64, "mixed": BYTES_PER_UNIT_MIXED,
             "mixed64": BYTES_PER_UNIT_MIXED64}[args.precision]
    name, (dms, dn) = max(prof.items(), key=lambda kv: kv[1][0])
    peaks, peak_kind = _load_peaks()
    roof = None
    if dn > 0 and name in table:
        units = cells if name == "predict" else act_mean
        bytes_per_launch = table[name] * units
        if name == "pcg_loop":
            # one launch runs every iteration of a solve
            iters2 = info2["iters_total"] / max(args.steps, 1)
            bytes_per_launch *= iters2 * args.steps / dn
        t_launch = dms * 1e-3 / dn
        if name == "predict" and args.precision == "fp64":
            flops = FLOPS_PER_CELL_FP64_PREDICT * cells
            achieved = flops / t_launch / 1e12
            peak = FP64_PEAK_GFLOPS / 1e3
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "kernel": "k_predict",
                    "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (FP64 pipe)",
                    "flops_per_launch": flops, "bytes_per_launch": bytes_per_launch,
                    "hbm_frac": bytes_per_launch / t_launch / 1e9 / peaks["hbm_gbs"],
                    "launches_per_step": dn / args.steps, "avg_launch_us": 1e6 * t_launch}
        else:
            achieved = bytes_per_launch / t_launch / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": f"k_{name}",
                    "peak_kind": peak_kind, "bytes_per_launch": bytes_per_launch,
                    "launches_per_step": dn / args.steps, "avg_launch_us": 1e6 * t_launch}

    # end to end through the C ABI with pinned host buffers, per step:
    # H2D of the step's input state, the step, D2H of its result
    e2e = None
    if args.e2e_steps > 0:
        n = cells
        hb = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(3)]
        G.get_state_ptr(hb[0].data_ptr(), hb[1].data_ptr(), hb[2].data_ptr())
        torch.cuda.synchronize()
        G.set_profiling(False)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            G.put_state_ptr(hb[0].data_ptr(), hb[1].data_ptr(), hb[2].data_ptr())
            G.step(wl.dt)
            G.get_state_ptr(hb[0].data_ptr(), hb[1].data_ptr(), hb[2].data_ptr())
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": ws * cells * args.e2e_steps / el, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * n, "d2h_bytes_per_step": 3 * 8 * n,
               "steps": args.e2e_steps}

    network = None
    if ws == 1 and args.form_steps > 0:
        network = time_network(wl, args)

    forms = None
    if ws == 1 and args.form_steps > 0:
        forms = compare_forms(wl, G, info2["last"]["t"], args)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle as O
        v, k, el = _oracle_sample(wl, args.cpu_steps, args.cpu_budget, O.CRIT_ETA_D)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"member 0 (50000 cells), {k} time steps from t = 0 ({el:.1f} s of one host "
                         f"thread), FP64 C oracle; the GPU's timed steps start at t = {args.t_start} s"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "members_per_gpu": len(wl.members),
                       "cells_per_member": wl.members[0].nx, "dt": wl.dt, "t_start": args.t_start,
                       "mode": args.mode, "precond": args.precond, "precision": args.precision,
                       "rtol": rtol, "l2": "per-step state > 129 MB L2 (154 MB FP64, 77 MB FP32 + FP64 operator); no flush",
                       "error_vs_oracle": ("max|d eta| <= 1e-9 a (tests/test_gpu_parity.py)" if args.precision == "fp64"
                                           else "max|d eta| <= 1e-4 a while masks agree (tests/test_gpu_mixed.py)"),
                       "mean_active_cells_per_step": act_mean, "mean_krylov_iters_per_step": iters_mean,
                       "spin_up_steps": n_spin, "spin_up_s": t_spin},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "timed_region": "nh_run replaying captured CUDA graphs (FP64) or step by step (mixed); "
                            "roofline and kernel times from a second, event-profiled pass of the same length",
            "clocks": clk,
            "kernel_ms": {k: v[0] for k, v in prof.items() if v[1] > 0},
            "kernel_launches": {k: v[1] for k, v in prof.items() if v[1] > 0},
            "forms": forms,
            "network": network,
        }
        print(json.dumps(out))
    G.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


# DG-P1 / LDG path (nhswe_dg.h): algorithmic bytes per unit (FP64).  Units:
# elements of the batch for the predictor and the compaction, marked elements
# for the rest (the cyclic reduction's and back-substitution's bytes are
# summed over their levels by _dg_cr_bytes).
BYTES_PER_UNIT_DG = {
    "predict": 129.0,   # read h, hu, hw, d0 at both nodes (64); write h~, hu~, hw~, p = 0 (64); the mark
    "compact": 6.0,     # read the mark, write the mask byte and the int32 list entry
    "local": 272.0,     # read list (8), h~, hu~, hw~, d0 at both nodes (64), outside hu (8); write hu(p) map,
                        # correction factors (14 doubles) and the row's own blocks (10 doubles)
    "form": 104.0,      # read list (8), left neighbour's hu_R map (32), D00, r0 (16); write L, D00, r0 (48)
    "correct": 368.0,   # read list, x (own + next), 14 local doubles, h~, hw~ (176); write hu, hw, p (48);
                        # residual check: the row (112) and both neighbours' x (32)
}


# The DG predictor is bound by the FP64 pipe: FP64 operations per element and
# step counted from the algorithm (a node: 1/h, u, three flux components and
# the wave speed, 11; an interface: the Rusanov flux, 19; an element: volume
# and interface terms through the inverse mass matrix and the nodal source,
# 39, the static slope 2; stage updates 12 and 18; two nodes and one
# interface per element and stage; criterion and mass 11): 205.
FLOPS_PER_ELEMENT_DG_PREDICT = 205.0


def _dg_cr_bytes(n0, ne, small_rows=512):
    """Algorithmic bytes of the block cyclic reduction of one member with n0
    marked elements (rows of 14 doubles, x of 2): (reduce incl. the
    shared-memory levels, back-substitution of the global levels)."""
    lev = 0
    while -(-ne // (1 << lev)) > small_rows:
        lev += 1
    red = back = 0.0
    n = n0
    for _ in range(lev):
        n1 = -(-n // 2)
        red += 112.0 * n + 112.0 * n1          # read every row of the level, write the even ones
        back += 112.0 * (n - n1) + 16.0 * n1 + 16.0 * n   # odd rows and x of the level above in, x out
        n = n1
    red += 112.0 * n + 16.0 * n                # k_cr_small: rows in, x out
    return red, back


def run_dg(args):
    """--workload dg_1d: the paper's own discretisation (DG-P1 predictor, LDG
    mixed solve) on a batch of 1D slides, 64 members x 50 000 elements
    (1e5 nodes each), adaptive |eta/d| > 1e-3 with one enlarging element,
    FP64; timed after a spin-up to --t-start."""
    import torch
    from paper_2505_17025_gb300 import nhswe as N
    from paper_2505_17025_gb300 import workloads as W
    import oracle as O
    import oracle.oracle_dg as D

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    wl = W.slide_dg_1d(n_members=args.members, seed0=rank_seed0(args.members, rank))
    ms_ = wl.members
    m0 = ms_[0]
    ne, nb = m0.ne, len(ms_)
    G = N.GridDG(ne, m0.dx, np.stack([m.d0() for m in ms_]), nbatch=nb, x0=m0.xl)
    G.set_bottom_motion([dict(shape=m.slide, A=m.A, L=m.L, xc0=m.xc0, s0=m.s0, t0=m.t0) for m in ms_])
    crit = N.NH_CRIT_GLOBAL if args.mode == "global" else N.NH_CRIT_ETA_D
    G.set_criterion(crit, 1e-3, 1, False)
    G.set_state(np.stack([m.h for m in ms_]), np.stack([m.hu for m in ms_]), np.stack([m.hw for m in ms_]), 0.0)
    elements = ne * nb
    dt = wl.dt

    n_spin = int(round(args.t_start / dt))
    t_spin0 = time.perf_counter()
    if n_spin:
        st, _ = G.run(dt, n_spin)
        assert st == N.NH_OK, st
    t_spin = time.perf_counter() - t_spin0
    st, _ = G.run(dt, args.warmup)
    assert st == N.NH_OK, st
    # the timed window's start, handed to the oracle afterwards
    h0, hu0, hw0, _ = G.get_state()
    t_win = (n_spin + args.warmup) * dt

    stream = G.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.profiler.start()
    e0.record(stream)
    st, info = G.run(dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    assert st == N.NH_OK, st
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    h1, hu1, hw1, _ = G.get_state()
    ms = max_over_ranks(ms, ws, "cuda")
    value = ws * elements * args.steps / (ms * 1e-3)
    act_mean = info["active_total"] / max(args.steps, 1)

    G.set_profiling(True)
    st2, info2 = G.run(dt, args.steps)
    prof = G.get_profile()
    G.set_profiling(False)
    launches = sum(n for _, n in prof.values())

    # roofline of the dominant kernel class (bytes per launch / mean launch time)
    name, (dms, dn) = max(prof.items(), key=lambda kv: kv[1][0])
    peaks, peak_kind = _load_peaks()
    act_member = act_mean / nb
    red_b, back_b = _dg_cr_bytes(int(round(act_member)), ne)
    per_step = {"predict": BYTES_PER_UNIT_DG["predict"] * elements, "compact": BYTES_PER_UNIT_DG["compact"] * elements,
                "local": BYTES_PER_UNIT_DG["local"] * act_mean, "form": BYTES_PER_UNIT_DG["form"] * act_mean,
                "correct": BYTES_PER_UNIT_DG["correct"] * act_mean, "reduce": red_b * nb, "back": back_b * nb}
    roof = None
    if dn > 0 and name in per_step:
        launches_per_step = dn / args.steps
        bytes_per_launch = per_step[name] / launches_per_step
        t_launch = dms * 1e-3 / dn
        if name == "predict":
            flops = FLOPS_PER_ELEMENT_DG_PREDICT * elements
            achieved = flops / t_launch / 1e12
            peak = FP64_PEAK_GFLOPS / 1e3
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "kernel": "k_dg_predict",
                    "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (FP64 pipe)",
                    "flops_per_launch": flops, "bytes_per_launch": bytes_per_launch,
                    "hbm_frac": bytes_per_launch / t_launch / 1e9 / peaks["hbm_gbs"],
                    "launches_per_step": launches_per_step, "avg_launch_us": 1e6 * t_launch}
        else:
            achieved = bytes_per_launch / t_launch / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": f"k_dg_{name}",
                    "peak_kind": peak_kind, "bytes_per_launch": bytes_per_launch,
                    "launches_per_step": launches_per_step, "avg_launch_us": 1e6 * t_launch}
    step_bytes = sum(per_step.values())

    # error against the oracle on the timed window: members 0 and nb-1 handed
    # over at the window's start, the same steps on the oracle
    errs, cpu = [], None
    t_or = 0.0
    if rank == 0 and not args.no_cpu_baseline:
        for b in sorted({0, nb - 1})[:max(1, args.err_members)]:
            m = ms_[b]
            p = D.ParamsDG(ne=ne, dx=m.dx, xl=m.xl, b0=m.b0, b1=m.b1, slide=m.slide, A=m.A, L=m.L, xc0=m.xc0,
                           s0=m.s0, t0=m.t0, crit=O.CRIT_GLOBAL if args.mode == "global" else O.CRIT_ETA_D,
                           knh=1e-3, enlarge=1)
            s = D.StateDG(h0[b], hu0[b], hw0[b])
            tt = time.perf_counter()
            for k in range(args.steps):
                t = t_win + k * dt
                st_o, _ = D.step(p, t, n_spin + args.warmup + k, dt, s)
                assert st_o == O.OK
            t_or += time.perf_counter() - tt
            scale_u = m.A * math.sqrt(9.81 * (m.b0 + m.b1 * ne * m.dx))
            errs.append({"member": b, "max_deta_over_a": float(np.max(np.abs(h1[b] - s.h)) / m.A),
                         "max_dhu_over_a_sqrt_gh": float(np.max(np.abs(hu1[b] - s.hu)) / scale_u),
                         "max_dhw_over_a_sqrt_gh": float(np.max(np.abs(hw1[b] - s.hw)) / scale_u)})
        n_or = len(errs) * args.steps
        cpu = {"value": ne * n_or / t_or, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(errs)} member(s) of {ne} elements, the timed window's {args.steps} steps each "
                         f"({t_or:.1f} s of one host thread), FP64 C DG oracle (banded LDG solve, 2 refinements)"}

    e2e = None
    if args.e2e_steps > 0:
        t_now = info2["last"]["t"]
        hb = [np.empty((nb, 2 * ne)) for _ in range(4)]
        h, hu, hw, _ = G.get_state()
        torch.cuda.synchronize()
        tt = time.perf_counter()
        for k in range(args.e2e_steps):
            G.set_state(h, hu, hw, t_now + k * dt)
            G.step(dt)
            h, hu, hw, _ = G.get_state()
        el = time.perf_counter() - tt
        e2e = {"value": ws * elements * args.e2e_steps / el, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * 2 * elements, "d2h_bytes_per_step": 4 * 8 * 2 * elements,
               "steps": args.e2e_steps}

    if rank == 0:
        out = {
            "metric": "element-updates/s of the DG-P1 / LDG step incl. the LDG solve", "value": value,
            "unit": "element-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"DG-P1/LDG 1D slides, {nb} members x {ne} elements, adaptive |eta/d|>1e-3 "
                                   f"+ 1-element enlargement" if args.mode != "global" else
                                   f"DG-P1/LDG 1D slides, {nb} members x {ne} elements, global",
                       "dt": dt, "t_start": t_win, "spin_up_steps": n_spin, "spin_up_s": t_spin,
                       "mean_marked_elements_per_step": act_mean, "step_bytes_algorithmic": step_bytes,
                       "l2": "state (4 FP64 fields x 2 nodes) 205 MB per buffer > 129 MB L2; no flush",
                       "error_vs_oracle": errs},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "timed_region": "nh_dg_run replaying captured CUDA graphs; kernel times from a second, "
                            "event-profiled pass of the same length",
            "clocks": clk,
            "kernel_ms": {k: v[0] for k, v in prof.items() if v[1] > 0},
            "kernel_launches": {k: v[1] for k, v in prof.items() if v[1] > 0},
        }
        print(json.dumps(out))
    G.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="landslide_ensemble_2d",
                    choices=["landslide_ensemble_2d", "landslide_2d", "line_soliton_2d", "slide_1d",
                             "paper_ratios", "dg_1d"])
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed", "mixed64"],
                    help="fp64; mixed64 = FP32 state with the FP64 solve; mixed = FP32 Krylov in FP64 "
                         "refinement (1D only).  Default: fp64 (1D), mixed64 (2D)")
    ap.add_argument("--mode", default="adaptive", choices=["adaptive", "global"])
    ap.add_argument("--precond", default=None, choices=["line", "none", "mg"],
                    help="1D: line (default) or none; 2D: mg (default) or line")
    ap.add_argument("--t-start", type=float, default=0.5, help="1D: spin-up to this time (s)")
    ap.add_argument("--spin-steps", type=int, default=200, help="2D: untimed steps before the warm-up")
    ap.add_argument("--rtol", type=float, default=None,
                    help="2D: relative residual at which the timed form's solve stops (default: 1e-12 with "
                         "the FP64 state, 1e-9 with the FP32 state)")
    ap.add_argument("--knh", type=float, default=None, help="criterion threshold of the 2D workloads (default 1e-3)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=None)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--members", type=int, default=64, help="1D: members per GPU")
    ap.add_argument("--err-members", type=int, default=2, help="2D: members checked against the oracle")
    ap.add_argument("--ens-members", type=int, default=32, help="2D ensemble: members (32 in the workload)")
    ap.add_argument("--form-steps", type=int, default=None, help="timed steps per form (0: skip the comparison)")
    ap.add_argument("--form-harvest", type=int, default=20)
    ap.add_argument("--form-train", type=int, default=200)
    args = ap.parse_args()
    two_d = args.workload not in ("slide_1d", "paper_ratios", "dg_1d")
    if args.precision is None:
        args.precision = "mixed64" if two_d else "fp64"
    if args.precond is None:
        args.precond = "mg" if two_d else "line"
    if args.rtol is None:
        args.rtol = RTOL_FP32_STATE if args.precision == "mixed64" else 1e-12
    if args.e2e_steps is None:
        args.e2e_steps = 5 if two_d else 20
    if args.cpu_steps is None:
        args.cpu_steps = 2 if two_d else 400
    if args.form_steps is None:
        args.form_steps = 10 if two_d else 30
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.workload == "paper_ratios":
        run_paper_ratios(args)
    elif args.workload == "dg_1d" and args.impl == "ours":
        run_dg(args)
    elif args.impl == "reference":
        run_reference_2d(args) if two_d else run_reference(args)
    elif two_d:
        run_2d(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
