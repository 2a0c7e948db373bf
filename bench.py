"""Benchmark of the CGKS-5 S2O4 step on GB300 (one JSON line on rank 0).

Metric: cell-updates/s per S2O4 step (cells x steps / time) on the 3-D
Taylor-Green vortex (Ma 0.1, Re 1600, Pr 0.72, gamma 1.4) on a periodic
uniform [0, 2 pi]^3 mesh, 128^3 by default, in the fastest form that keeps
parity with the FP64 oracle at the FP64 bars: FP64 storage and arithmetic
with the interior interface flux in paired FP32 (--form pair, the default);
plain FP64 throughout (--form fp64) is timed beside it from the same state,
and so are the FP32 form, the learned selector and the batched ensemble.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload tgv128|tgv256|tgv64|vortex64] [--form pair|fp64]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

A step is one full S2O4 step (time-step reduction, two stages of
reconstruction + interface flux + update) over the whole mesh.  The state
(1.3 GB at 128^3) is larger than the 129 MB L2, so no flush is needed between
steps.  For N > 1 (torchrun) every rank advances an independent replica
(the path needs no exchange on one GPU per replica): weak scaling.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "tgv128": dict(dim=3, n=(128, 128, 128), desc="3-D Taylor-Green vortex 128^3, Ma 0.1, Re 1600, Pr 0.72, FP64"),
    "tgv256": dict(dim=3, n=(256, 256, 256), desc="3-D Taylor-Green vortex 256^3, Ma 0.1, Re 1600, Pr 0.72, FP64"),
    "tgv64": dict(dim=3, n=(64, 64, 64), desc="3-D Taylor-Green vortex 64^3 (profiling size), Ma 0.1, Re 1600, FP64"),
    "vortex64": dict(dim=2, n=(64, 64), desc="2-D isentropic vortex 64^2 over [0,10]^2, eps 5"),
}

# Algorithmic FP64 (or FP32) flops per unit of work, recounted from the
# kernels' source by tests/flop_count.cpp (the device routines built for the
# host with a value-numbering compute type: shared subexpressions once,
# products with exact 0 or +-1 and sums with exact 0 not at all, only what
# a stored result depends on; +, -, * and / one flop, FMA two; special
# functions not counted) and pinned by tests/test_flop_count.py.  Flux: per
# face Gauss point, keyed by (kernel, dim, viscous); the viscous form adds
# the collision-time and Prandtl-fix terms.  The same algorithm runs in the
# FP64, FP32 and paired forms.
ALG_FLOPS_PER_UNIT = {
    ("flux", 3, True): 2919.0,
    ("flux", 2, True): 1672.0,
    ("flux", 2, False): 766.0,
}
# Executed work per unit from ncu instruction counts (TGV 64^3, same
# kernels): 2 DFMA + DADD + DMUL (FP64) or 2 FFMA + FADD + FMUL (FP32),
# which includes the instruction sequences of divisions and special
# functions and whatever the compiler recomputes.  The FP64 reconstruction
# is not listed: since its FP32 screen of the smoothness indicators its FP64
# work per cell depends on the data.
EXEC_FLOPS_PER_UNIT = {
    ("flux", 3): 3.616e3,
}
# the paired form's flux (ncu, TGV 64^3, profiles/flux_pair_tgv64_full.md):
# FP32 flops it executes per face Gauss point for its FP64-equivalent work
# (2 FFMA + FADD + FMUL; plus 101 FP64 flops of conversions)
EXEC_FP32_FLOPS_PER_UNIT_PAIR = {
    ("flux", 3): 26580.0,
}
# DRAM bytes per face point of the three flux kernels as built (inputs
# staged as TMA tiles), from one launch-level capture at TGV 64^3
# (profiles/flux_dram_tgv64.md; read + write averaged over the launches)
DRAM_BYTES_PER_UNIT_PAIR = {
    ("flux", 3): (1.0079e9 + 0.7331e9) / (262144 * 12),
}
# DRAM bytes per unit of the same capture (read + write), for `traffic`
DRAM_BYTES_PER_UNIT = {
    ("flux", 3): (1.0084e9 + 0.7103e9) / (262144 * 12),
}
# the same for the FP32 form (update: per (cell, variable))
EXEC_FLOPS_PER_UNIT_FP32 = {
    ("recon", 3): 1.262e4,
    ("flux", 3): 3.395e3,
    ("update", 3): 158.0,
}
DRAM_BYTES_PER_UNIT_FP32 = {
    ("recon", 3): (151.1e6 + 465.3e6) / 262144,
    ("flux", 3): (503.4e6 + 333.5e6) / (262144 * 12),
    ("update", 3): (388.5e6 + 159.3e6) / (262144 * 5),
}


# kernels launched per S2O4 step: time-step reduction (reset, FP32 screen,
# FP64 rate of the candidates, final), two stages x (reconstruction,
# interface flux, update), time advance
KERNELS_PER_STEP = 4 + 2 * 3 + 1


def mesh_kwargs(wl):
    if wl.startswith("tgv"):
        return dict(lo=(0.0, 0.0, 0.0), hi=(2 * math.pi,) * 3, mu=1.0 / 1600.0, prandtl=0.72, tau_mode=2, cfl=0.5)
    return dict(lo=(0.0, 0.0), hi=(10.0, 10.0), tau_mode=0, cfl=0.5)


def field_fn(wl):
    import synth
    if wl.startswith("tgv"):
        return lambda x, y, z: synth.taylor_green_3d(x, y, z, mach=0.1)
    return lambda x, y: synth.isentropic_vortex_2d(x, y)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for line in out.stdout.strip().splitlines():
                    self.rows.append([x.strip() for x in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._th.join(timeout=10)

    def summary(self):
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for i, nme in enumerate(names):
                    if r[5 + i].lower() == "active":
                        reasons.add(nme)
            except (ValueError, IndexError):
                continue
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def fp64_alu_peak_tflops(sm_count=152, sm_mhz=2070.0):
    """FP64 FMA pipe peak from unit counts and clock: 2 FP64 FMA per clock per SM
    on GB300 (the probe of this project measured 1.19-1.20 TFLOP/s, 95% of it)."""
    return sm_count * 2 * 2 * sm_mhz * 1e6 / 1e12


def fp32_alu_peak_tflops(sm_count=152, sm_mhz=2070.0):
    """FP32 FMA pipe peak: 128 FP32 FMA per clock per SM (a probe of this
    project measured 72.9-73.3 TFLOP/s)."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def step_hbm(ncell, dim, ms_per_step, peak_gbs):
    """The step's share of HBM bandwidth on the algorithmic bytes of an S2O4
    step: six state-sized transfers per cell (stage 1 reads U^n and writes
    U* and the stash; stage 2 reads U* and the stash and writes U^{n+1}),
    the FP64 state being (dim + 2) variables x (1 + dim + lines) fields.
    A step-level figure: the sweep is bound by its arithmetic, so this is
    small by design."""
    nf = 1 + dim + (12 if dim == 3 else 4)
    per_cell = 6 * 8 * (dim + 2) * nf
    gbs = ncell * per_cell / (ms_per_step * 1e-3) / 1e9
    return {"algorithmic_bytes_per_cell": per_cell, "achieved_gbs": gbs, "peak_gbs": peak_gbs,
            "frac": (gbs / peak_gbs) if peak_gbs else None}


def roofline(prof, spec, ncell, precision, viscous):
    """Roofline of the dominant kernel of a timed form: its algorithmic flops
    per unit (ALG_FLOPS_PER_UNIT) times the units of one launch, over its
    average CUDA-event launch time, against the ALU pipe peak of its
    precision; the executed (ncu) count gives frac_executed beside it."""
    name, (launches, tot_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    avg_ms = tot_ms / max(launches, 1)
    dim = spec["dim"]
    if name == "update":
        units = ncell * (dim + 2)
    elif name in ("recon", "dt"):
        units = ncell
    else:
        units = ncell * dim * (4 if dim == 3 else 2)
    exe = (EXEC_FLOPS_PER_UNIT if precision != 1 else EXEC_FLOPS_PER_UNIT_FP32).get((name, dim))
    dram = (DRAM_BYTES_PER_UNIT if precision == 0 else DRAM_BYTES_PER_UNIT_FP32 if precision == 1
            else DRAM_BYTES_PER_UNIT_PAIR)
    alg = ALG_FLOPS_PER_UNIT.get((name, dim, viscous))
    if precision == 1:
        peak = fp32_alu_peak_tflops()
        src = ("FP32 FMA pipe: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz, derived (an FMA-chain probe measured "
               "72.9-73.3 TFLOP/s)")
    else:
        peak = fp64_alu_peak_tflops()
        src = ("FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz, derived (an FMA-chain probe measured "
               "1.19-1.20 TFLOP/s)")
        if precision == 2:
            src += "; the paired form's flux runs its FP64-equivalent work on the FP32 pipe"
    sec = avg_ms / 1e3
    out = {"bound": "alu", "kernel": name, "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
           "traffic": None, "avg_launch_ms": avg_ms, "units_per_launch": units, "peak_source": src}
    if alg:
        achieved = alg * units / sec / 1e12
        out.update({"achieved": achieved, "frac": achieved / peak, "flops_per_unit": alg,
                    "flops_per_launch": alg * units,
                    "flops_source": "algorithmic count of the kernel's source (tests/flop_count.cpp)"})
    if exe and precision != 2:
        out.update({"flops_per_unit_executed": exe, "frac_executed": exe * units / sec / 1e12 / peak})
    pair32 = EXEC_FP32_FLOPS_PER_UNIT_PAIR.get((name, dim)) if precision == 2 and name == "flux" else None
    if pair32:
        p32 = fp32_alu_peak_tflops()
        out.update({"fp32_flops_per_unit_executed": pair32, "frac_fp32_pipe": pair32 * units / sec / 1e12 / p32,
                    "note": "FP64-equivalent work delivered through the FP32 pipe in paired arithmetic: frac is "
                            "against the FP64 pipe it replaces and can exceed 1; frac_fp32_pipe is the FP32 "
                            "pipe's own use"})
    dbu = dram.get((name, dim))
    if dbu:
        out.update({"traffic": dbu * units,
                    "traffic_source": "ncu dram__bytes_read+write of a 64^3 capture, scaled by units"})
    if not alg:
        out["note"] = "flops per unit not counted for this kernel"
    return out


def cpu_baseline(wl, sample_cells=None):
    """Time the CPU oracle, as it stands, on a bounded sample of the workload:
    the same analytic field and physics on a smaller periodic mesh (same
    per-cell work), whole S2O4 steps."""
    import oracle.oracle as o
    spec = WORKLOADS[wl]
    dim = spec["dim"]
    kw = mesh_kwargs(wl)
    if dim == 3:
        m = sample_cells or 40
        n = (m, m, m)
    else:
        n = (64, 64)
    orc = o.Oracle(dim, n, **kw)
    orc.init(field_fn(wl))
    orc.step(1)  # warm-up (builds tables, touches memory)
    steps = 3 if dim == 3 else 20
    t0 = time.perf_counter()
    orc.step(steps)
    el = time.perf_counter() - t0
    ncell = int(math.prod(n))
    threads = o.set_threads(0)
    out = {"value": ncell * steps / el, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
           "sample": "%s on %s (%d cells, same per-cell work), %d S2O4 steps, %.1f s" % (
               spec["desc"].split(",")[0], "x".join(map(str, n)), ncell, steps, el)}
    # the same on one core, on a smaller sample
    n1 = (12, 12, 12) if dim == 3 else (32, 32)
    o1 = o.Oracle(dim, n1, **kw)
    o1.init(field_fn(wl))
    o.set_threads(1)
    try:
        o1.step(1)
        steps1 = 2 if dim == 3 else 10
        t0 = time.perf_counter()
        o1.step(steps1)
        el1 = time.perf_counter() - t0
    finally:
        o.set_threads(threads)
    nc1 = int(math.prod(n1))
    out["single_core"] = {"value": nc1 * steps1 / el1, "unit": "cell-updates/s", "cores": 1,
                          "sample": "%s cells, %d S2O4 steps, %.1f s" % ("x".join(map(str, n1)), steps1, el1)}
    return out


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle timed on the host cores."""
    if rank != 0:
        return 0
    wl = args.workload
    spec = WORKLOADS[wl]
    import oracle.oracle as o
    dim = spec["dim"]
    kw = mesh_kwargs(wl)
    n = (20, 20, 20) if dim == 3 else (64, 64)
    orc = o.Oracle(dim, n, **kw)
    orc.init(field_fn(wl))
    for _ in range(args.warmup):
        orc.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.step(1)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    ncell = int(math.prod(n))
    val = ncell * args.steps / tot
    threads = o.set_threads(0)
    line = {
        "impl": "reference", "metric": "cell-updates/s per S2O4 step", "value": val, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl, "description": spec["desc"], "sample_mesh": "x".join(map(str, n)),
                   "note": "CPU oracle (plain FP64 C, OpenMP) on a bounded sample of the workload"},
        "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
                         "sample": "%s cells, %d steps" % ("x".join(map(str, n)), args.steps)},
        "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def e2e_overlapped(make_mesh, h_in, outs, nsteps):
    """End to end through the public API with two contexts on two streams,
    driven from one host thread: each step copies its state in from
    page-locked host memory, advances one S2O4 step and copies the new state
    out.  The copies are enqueued without waiting (cgks_set_state_async,
    cgks_get_state_async), so one context's copies run on the copy engines
    while the other context's step runs on the SMs.  Returns the wall time in
    seconds, both streams drained; outs[i] holds lane i's last result."""
    import torch
    from paper_2508_08965_gb300 import CgksError
    lanes = []
    try:
        for _ in range(2):
            lanes.append(make_mesh(torch.cuda.Stream()))
    except CgksError as err:
        if err.status != -2:  # CGKS_ENOMEM: two contexts do not fit in device memory
            raise
        for m in lanes:
            m.close()
        return None
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the first lane's copy alone (the fill), then the second lane's copy
        # overlapping the first lane's step, and so on
        lanes[0].set_state_async(h_in, 0.0)
        lanes[0].sync()
        if nsteps > 1:
            lanes[1].set_state_async(h_in, 0.0)
        for i in range(nsteps):
            m = lanes[i % 2]
            m.step(1)
            m.get_state_async(outs[i % 2])
            if i + 2 < nsteps:
                m.set_state_async(h_in, 0.0)
        for m in lanes:
            m.sync()
        el = time.perf_counter() - t0
    finally:
        for m in lanes:
            m.close()
    return el


def ensemble_bench(args, stream, ncase=256):
    """The batched ensemble: ncase seeded 2-D cases of uneven size (vortex or
    four-quadrant Riemann), FP32 form.  The batch (autotuned tiles, one graph
    launch per K steps) against the same cases as sequential single-case
    contexts, one cgks_step call each; both from the same states, same steps."""
    import numpy as np
    import torch
    import synth
    from paper_2508_08965_gb300 import Batch, CgksError, Mesh
    # The plain method has no positivity guarantee: some random four-quadrant
    # draws turn non-physical within a few steps (the oracle fails on the same
    # draws).  Each Riemann draw is run once, alone, for every step the bench
    # takes; a draw that fails is replaced by the next one of the stream.
    need = 2 * args.warmup + 3 * args.steps + 2
    specs, rejected = [], []
    for sp in synth.ensemble_stream():
        if sp["kind"] == "riemann":
            m = Mesh(precision=1, stream=stream, **synth.spec_mesh(sp))
            m.init(synth.spec_field(sp))
            try:
                m.step(need)
            except CgksError:
                rejected.append(sp["seed"])
                continue
            finally:
                m.close()
        specs.append(sp)
        if len(specs) == ncase:
            break
    kws = [synth.spec_mesh(sp) for sp in specs]
    b = Batch(kws, precision=1, stream=stream)
    meshes, init_states = [], {}
    for k, sp in enumerate(specs):
        m = Mesh(precision=1, stream=stream, **kws[k])
        m.init(synth.spec_field(sp))
        st = torch.empty(b.state_shape(k), dtype=torch.float64, device="cuda")
        m.get_state(out=st)
        b.set_state(k, st)
        if k % max(1, ncase // 16) == 0:
            init_states[k] = st.cpu().numpy()
        meshes.append(m)
    t0 = time.perf_counter()
    tiles, tune_ms = b.tune(reps=3)
    tune_s = time.perf_counter() - t0
    for m in meshes:
        m.step(args.warmup)
    b.step(args.warmup)
    b.step(args.steps)  # captures the graph of K steps (untimed)
    # restart both arms from the states after warm-up plus K steps: time K more
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for m in meshes:
        m.step(args.steps)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    e0.record(stream)
    for m in meshes:
        m.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    worst = 0.0
    sampled = list(range(0, ncase, max(1, ncase // 16)))
    for k in sampled:
        sb, _ = b.get_state(k)
        ss, _ = meshes[k].get_state()
        worst = max(worst, float(np.abs(sb - ss).max() / max(np.abs(ss).max(), 1e-300)))
    # how far rounding alone carries these problems: the same single-case
    # runs from initial states moved by one unit in the last place
    rng = np.random.default_rng(7)
    sens = 0.0
    for k in sampled:
        s0 = init_states[k]
        m = Mesh(precision=1, stream=stream, **kws[k])
        m.set_state(s0 * (1 + rng.choice([-1.0, 1.0], size=s0.shape) * 2.0 ** -53), 0.0)
        m.step(args.warmup + 2 * args.steps)
        sp, _ = m.get_state()
        m.close()
        ss, _ = meshes[k].get_state()
        sens = max(sens, float(np.abs(sp - ss).max() / max(np.abs(ss).max(), 1e-300)))
    ncell = int(b.ncell)
    for m in meshes:
        m.close()
    b.close()
    return {
        "workload": "%d 2-D cases, sizes from {64,128,256,512}^2, vortex or four-quadrant Riemann, FP32 form" % ncase,
        "cells": ncell, "steps": args.steps,
        "rejected_riemann_draws": len(rejected),
        "batched": {"value": ncell * args.steps / (ms_b / 1e3), "unit": "cell-updates/s",
                    "ms_per_step": ms_b / args.steps, "launch": "one CUDA graph per %d steps" % args.steps,
                    "tiles": tiles, "tune_s": tune_s},
        "sequential": {"value": ncell * args.steps / (ms_s / 1e3), "unit": "cell-updates/s",
                       "ms_per_step": ms_s / args.steps, "launch": "one cgks_step call per case"},
        "speedup": ms_s / ms_b,
        "max_rel_diff_batched_vs_sequential": worst,
        "max_rel_diff_sequential_one_ulp_input": sens,
        "sampled_cases": len(sampled),
        "clocks": clk.summary(),
    }


def selector_bench(args, stream, s_tgv_init=None, s_tgv_fp64=None):
    """The learned selector: held-out four-quadrant Riemann problems on
    1024^2, held-out shock-vortex interactions on 1024^2 cells of [0, 2] x
    [0, 1], and the TGV 128^3, each with and without the trained selector
    from the same initial state, in the FP32 form, and for one Riemann and
    the shock-vortex cases also in the plain FP64 form: time per step and per
    reconstruction, skip, fallback (full GENO) and low-confidence rates, and
    the density difference from the plain adaptive method."""
    import numpy as np
    import torch
    import synth
    from paper_2508_08965_gb300 import CgksError, Mesh, selector
    params, thr, lo = selector.load()
    out = {"thr_skip": thr, "thr_lo": lo, "cases": []}

    def run(kw, fn, s0, steps, on, precision, linear=False):
        m = Mesh(precision=precision, stream=stream, linear=linear, **kw)
        if s0 is None:
            m.init(fn)
        else:
            m.set_state(s0, 0.0)
        if on:
            m.set_selector(params, thr, lo)
        m.step(args.warmup)
        m.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        m.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = m.profile_read()
        stats = m.selector_stats() if on else (0, 0)
        s, _ = m.get_state()
        m.close()
        return s, e0.elapsed_time(e1) / steps, prof["recon"][1] / prof["recon"][0], stats

    cases = []
    for seed in (9001, 9002, 9003, 9004):
        st = synth.riemann4_params(seed)
        cases.append(("riemann1024 seed %d" % seed,
                      dict(dim=2, n=(1024, 1024), lo=(0, 0), hi=(1, 1), bc=[1, 1, 1, 1], tau_mode=1),
                      (lambda st: (lambda x, y: synth.riemann4_2d(x, y, st)))(st), None,
                      (1, 0) if seed == 9001 else (1,)))
    for seed in (9101, 9102):
        mach, eps = synth.shock_vortex_params(seed)
        cases.append(("shockvortex1024 mach %.2f eps %.2f" % (mach, eps),
                      dict(dim=2, n=(1024, 1024), lo=(0, 0), hi=(2, 1), bc=[4, 1, 2, 2], tau_mode=1,
                           bc_state=[synth.shock_vortex_inflow(mach)]),
                      (lambda mach, eps: (lambda x, y: synth.shock_vortex_2d(x, y, mach, eps)))(mach, eps), None,
                      (1, 0)))
    cases.append(("tgv128", dict(dim=3, n=(128, 128, 128), **mesh_kwargs("tgv128")), field_fn("tgv128"), s_tgv_init,
                  (1,)))
    runs = [(name if p == 1 else name + " fp64", kw, fn, s0, p) for name, kw, fn, s0, precs in cases for p in precs]
    for name, kw, fn, s0, precision in runs:
        try:
            s_plain, ms0, rc0, _ = run(kw, fn, s0, args.steps, False, precision)
            s_sel, ms1, rc1, (nskip, nuns) = run(kw, fn, s0, args.steps, True, precision)
        except CgksError as ex:
            out["cases"].append({"case": name, "error": str(ex)})
            continue
        try:  # the ceiling of any selector: every cell skips, for free (chi = 1, no features, no inference)
            _, msl, rcl, _ = run(kw, fn, s0, args.steps, False, precision, linear=True)
        except CgksError:
            msl = rcl = None
        ncell = int(np.prod(kw["n"]))
        recons = 2 * (args.warmup + args.steps) * ncell
        e = s_sel[0, 0] - s_plain[0, 0]
        rec = {"case": name, "form": "fp32" if precision == 1 else "fp64",
               "ms_per_step": {"plain": ms0, "selector": ms1, "skip_all_free": msl}, "speedup": ms0 / ms1,
               "speedup_ceiling": ms0 / msl if msl else None,
               "recon_ms": {"plain": rc0, "selector": rc1, "skip_all_free": rcl},
               "skip_rate": nskip / recons, "fallback_rate": 1.0 - nskip / recons,
               "low_confidence_rate": nuns / recons,
               "density_l2_vs_plain": float(np.sqrt(np.mean(e * e) / np.mean(s_plain[0, 0] ** 2))),
               "density_linf_vs_plain": float(np.abs(e).max() / np.abs(s_plain[0, 0]).max())}
        if name == "tgv128" and s_tgv_fp64 is not None:
            d = s_sel[0, 0] - s_tgv_fp64[0, 0]
            rec["density_l2_vs_fp64"] = float(np.sqrt(np.mean(d * d)))
            rec["value"] = ncell / (ms1 / 1e3)
        out["cases"].append(rec)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv128", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-selector", action="store_true")
    ap.add_argument("--form", default="pair", choices=["pair", "fp64"],
                    help="the headline FP64-parity form: pair (FP64 with the interior interface flux in paired "
                         "FP32, the default) or fp64 (FP64 throughout); the other is timed beside it")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2508_08965_gb300 import Mesh, replicas

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = args.workload
    spec = WORKLOADS[wl]
    viscous = mesh_kwargs(wl).get("mu", 0.0) > 0.0
    stream = torch.cuda.Stream()
    peaks = measured_peaks()

    def timed_form(precision, s0=None):
        """Warm up, then time K whole steps of one form on the context stream
        with per-kernel CUDA events; returns the mesh, its start state, the
        time, the per-kernel profile and the clock record."""
        mesh = Mesh(spec["dim"], spec["n"], stream=stream, precision=precision, **mesh_kwargs(wl))
        if s0 is None:
            mesh.init(field_fn(wl))
            s0 = mesh.get_state()[0]
        else:
            mesh.set_state(s0, 0.0)
        for _ in range(args.warmup):
            mesh.step(1)
        mesh.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            e0.record(stream)
            mesh.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        prof = mesh.profile_read()
        mesh.profile(False)
        return mesh, s0, replicas.job_time_ms(ms, device="cuda"), prof, clk

    head = 2 if args.form == "pair" else 0
    mesh, s_init, ms, prof, clk = timed_form(head)
    ncell = mesh.ncell
    flux_staging = ("TMA tiles (cp.async.bulk.tensor)" if mesh.flux_staging == "tma" else
                    "per-thread cp.async")
    value = replicas.whole_job_rate(ncell, args.steps, ms, world)

    # end to end through the C-ABI with host buffers: every step copies the
    # state in from pinned host memory, steps, and copies the new state out;
    # first one context waiting on each copy (serial), then two contexts whose
    # copies overlap each other's steps (the reported figure)
    shape = mesh.state_shape
    h_in = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    h_out = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    mesh.get_state(h_in.numpy())
    s_head = h_in.numpy().copy()  # the headline form's state after the warm-up and timed steps
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        mesh.set_state(h_in.numpy(), 0.0)
        mesh.step(1)
        mesh.get_state(h_out.numpy())
    torch.cuda.synchronize()
    e2e_s = replicas.job_time_ms(1e3 * (time.perf_counter() - t0), device="cuda") / 1e3
    state_bytes = int(np.prod(shape)) * 8
    mesh.close()
    outs = [torch.empty(shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    barrier()
    ov_s = e2e_overlapped(lambda st: Mesh(spec["dim"], spec["n"], stream=st, precision=head, **mesh_kwargs(wl)),
                          h_in, outs, args.e2e_steps)
    overlapped = ov_s is not None
    if overlapped:
        ov_s = replicas.job_time_ms(1e3 * ov_s, device="cuda") / 1e3
        lanes_match = all(np.array_equal(o.numpy(), h_out.numpy()) for o in outs[:min(2, args.e2e_steps)])
    else:
        ov_s, lanes_match = e2e_s, None
    kernels = {k: {"launches": v[0], "ms_total": v[1], "share": v[1] / max(sum(x[1] for x in prof.values()), 1e-30)}
               for k, v in prof.items()}

    # the other FP64-parity form from the same initial state and steps: the
    # plain FP64 state is the reference of every difference below (itself
    # parity-checked against the FP64 oracle)
    forms = {}
    other = 0 if head == 2 else 2
    mo, _, mso, profo, clko = timed_form(other, s_init)
    s_other, _ = mo.get_state()
    mo.close()
    s_fp64 = s_other if head == 2 else s_head
    s_pair = s_head if head == 2 else s_other
    ms_fp64 = mso if head == 2 else ms
    ms_pair = ms if head == 2 else mso
    e = s_pair - s_fp64
    forms["fp64"] = {
        "value": world * ncell * args.steps / (ms_fp64 / 1e3), "unit": "cell-updates/s",
        "ms_per_step": ms_fp64 / args.steps, "dtype": "f64",
        "note": "plain FP64 throughout",
    }
    forms["pair"] = {
        "value": world * ncell * args.steps / (ms_pair / 1e3), "unit": "cell-updates/s",
        "ms_per_step": ms_pair / args.steps, "speedup_vs_fp64": ms_fp64 / ms_pair,
        "dtype": "f64 storage and arithmetic; interior interface flux in paired f32 (hi + lo)",
        "difference_vs_fp64": {"steps": args.warmup + args.steps,
                               "density_linf": float(np.abs(e[0, 0]).max()),
                               "averages_linf_rel": float(np.abs(e[0]).max() / np.abs(s_fp64[0]).max())},
    }
    forms["fp64" if other == 0 else "pair"].update({
        "kernels": {k: {"launches": v[0], "ms_total": v[1]} for k, v in profo.items()},
        "roofline": roofline(profo, spec, ncell, other, viscous), "clocks": clko.summary()})
    if not args.no_fp32:
        m32, _, ms32, prof32, clk32 = timed_form(1, s_init)
        s32, _ = m32.get_state()
        m32.close()
        e = s32[0, 0] - s_fp64[0, 0]
        dim = spec["dim"]

        def ke(st):
            return float(np.mean(0.5 * (st[0, 1:1 + dim] ** 2).sum(axis=0) / st[0, 0]))

        forms["fp32"] = {
            "value": world * ncell * args.steps / (ms32 / 1e3), "unit": "cell-updates/s",
            "ms_per_step": ms32 / args.steps, "speedup_vs_fp64": ms_fp64 / ms32,
            "dtype": "f32 reconstruction/flux/weights/derivative fields; f64 averages, accumulation, metrics",
            "error_vs_fp64": {"steps": args.warmup + args.steps,
                              "density_l2": float(np.sqrt(np.mean(e * e))),
                              "density_linf": float(np.abs(e).max()),
                              "kinetic_energy_rel": abs(ke(s32) - ke(s_fp64)) / ke(s_fp64)},
            "kernels": {k: {"launches": v[0], "ms_total": v[1]} for k, v in prof32.items()},
            "roofline": roofline(prof32, spec, ncell, 1, viscous),
            "clocks": clk32.summary(),
        }

    line = {
        "metric": "cell-updates/s per S2O4 step", "value": value, "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32x2" if head == 2 else "f64", "data": "synthetic",
        "config": {"workload": wl, "description": spec["desc"], "cells": ncell,
                   "form": ("FP64 storage and arithmetic, interior interface flux in paired FP32 (hi + lo, about "
                            "48 bits); parity with the FP64 oracle at the FP64 bars" if head == 2 else
                            "FP64 throughout"),
                   "l2": "state (%.2f GB) larger than L2; no flush" % (state_bytes / 1e9),
                   "flux_staging": flux_staging,
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": world * ncell * args.e2e_steps / ov_s, "unit": "cell-updates/s",
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes, "steps": args.e2e_steps,
                "method": ("two contexts on two streams from one host thread; per step: state in from pinned "
                           "host memory (cgks_set_state_async), one S2O4 step (cgks_step), state out "
                           "(cgks_get_state_async); one context's copies overlap the other's step" if overlapped
                           else "one context (two do not fit in device memory); per step cgks_set_state, "
                                "cgks_step, cgks_get_state, each waiting"),
                "lanes_match_serial": lanes_match,
                "serial": {"value": world * ncell * args.e2e_steps / e2e_s, "unit": "cell-updates/s",
                           "method": "one context; cgks_set_state, cgks_step, cgks_get_state, each waiting"}},
        "gpu_launches": args.steps * KERNELS_PER_STEP,
        "kernels": kernels,
        "roofline": roofline(prof, spec, ncell, head, viscous),
        "clocks": clk.summary(),
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
        "hbm_step": step_hbm(ncell, spec["dim"], ms / args.steps, peaks.get("hbm_gbs")),
        "forms": forms,
    }
    if not args.no_selector:
        tgv128 = wl == "tgv128"  # the selector's TGV case starts from this run's state only at 128^3
        line["selector"] = selector_bench(args, stream, s_init if tgv128 else None, s_fp64 if tgv128 else None)
        tg = [c for c in line["selector"]["cases"] if c["case"] == "tgv128" and "value" in c]
        if tg and "fp32" in forms:
            forms["fp32_learned"] = {"value": tg[0]["value"], "unit": "cell-updates/s",
                                     "ms_per_step": tg[0]["ms_per_step"]["selector"],
                                     "speedup_vs_fp64": (ms_fp64 / args.steps) / tg[0]["ms_per_step"]["selector"],
                                     "density_l2_vs_fp64": tg[0].get("density_l2_vs_fp64"),
                                     "skip_rate": tg[0]["skip_rate"]}
    if not args.no_ensemble:
        line["ensemble"] = ensemble_bench(args, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(wl)
        except Exception as ex:  # the oracle is a reported baseline only
            line["cpu_baseline"] = {"error": str(ex)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0

if __name__ == "__main__":
    sys.exit(main())
