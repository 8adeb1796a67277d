#!/usr/bin/env python
"""Benchmark: PISO time steps of the 3-D lid-driven cavity on one GB300.

Default workload (the line's value): the 100^3 = 1M-cell cavity (unit cube,
lid u = 1, nu = 0.01, dt = 0.002, 2 pressure correctors, pressure CG to 1e-6
relative residual, FP64), cells permuted with seed 1234 and renumbered by
reverse Cuthill-McKee.  One "step" is one full PISO time step: momentum
assembly, three BiCGStab momentum solves, and two pressure corrections (H/A,
pressure assembly, Jacobi-PCG, flux and velocity correction).

The same line carries, as extra keys, the other benchmark configurations
timed the same way: the 200^3 = 8M-cell cavity (``cavity3d_200``: FP64 and
mixed-precision pressure solves, its stated 20 steps) and the batch of 256
cavities (``batch256``: FP64 and mixed, against a per-case loop of the
single-case solver over the same number of steps); per-stage effective
bandwidth of the assembly and correction kernels; the paper's Table 3
operator ratios; bytes per cell against the paper's 540.

The timed steps start from rest, after W untimed warm-up steps on the same
case; L2 is flushed (256 MiB write) between timed steps, outside the timed
windows.  Device time is taken with CUDA events on the library's stream.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle (its
OpenMP build on all host cores) on the same workload: the first three PISO
steps from rest.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PISO steps/s & cell-updates/s; pressure-CG HBM GB/s vs peak; mixed vs FP64"
UNIT = "cell-updates/s"

BATCH = dict(n_cases=256, seed=7, dt=0.002, n_corr=2)

WORKLOADS = {
    "cavity3d_100": dict(n=100, dim=3, nu=0.01, dt=0.002, n_corr=2, seed=1234),
    "cavity3d_200": dict(n=200, dim=3, nu=0.01, dt=0.001, n_corr=2, seed=1234),
    # larger than L2, small enough for an ncu capture: the CG's global-memory forms
    "cavity3d_130": dict(n=130, dim=3, nu=0.01, dt=0.002, n_corr=2, seed=1234),
    "cavity3d_40": dict(n=40, dim=3, nu=0.01, dt=0.002, n_corr=2, seed=1234),
    "cavity2d_20": dict(n=20, dim=2, nu=0.1, dt=0.005, n_corr=2, seed=None),
    # transient Poiseuille flow, 3200 x 300 2-D pipe, inlet 0.01 sin(pi t)
    "tp1M": dict(tp=True, nu=3.3e-6, dt=1e-4, n_corr=2),
    "batch256": dict(batch=True),
}
# PISO steps from rest the CPU reference arm times on the workload itself
REF_STEPS = 3

# ncu DRAM traffic (read + write bytes) per k_pcg launch, measured on the
# workload named here; valid only for the kernel source it was taken on
PCG_TRAFFIC = {"source_sha1": "94879bea0e5c65de63ce5b00ad048c7627d66eec", "bytes_per_iter": 547934,
               "workload": "cavity3d_100", "capture": "second pressure solve of the first step (789 iterations)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_mesh(w):
    import meshgen as mg
    if w.get("tp"):
        return mg.tp_channel()
    if w["dim"] == 2:
        return mg.cavity2d(w["n"])
    m = mg.cavity3d(w["n"])
    if w["seed"] is not None:
        m = mg.permute_cells(m, mg.random_permutation(m.n_cells, w["seed"]))
    return m


def ref_cell(w, m):
    """Pressure reference: the corner cell of a closed cavity; none when an
    outlet fixes p."""
    return -1 if w.get("tp") else m.corner_cell


def set_bc(L, case_h, w, m, k):
    """Time-dependent boundary values before step k (0-based, from rest):
    the tp1M inlet at the new time level (k + 1) dt."""
    if not w.get("tp"):
        return
    import meshgen as mg
    u = (ctypes.c_double * 3)(*mg.tp_inlet((k + 1) * w["dt"]))
    _check_rc(L.fv_patch_set_value(case_h, m.patch("inlet"), u, 0.0), "fv_patch_set_value")


def _check_rc(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with status {rc}")


def workload_name(name, w, m):
    if w.get("tp"):
        return (f"{name}: transient Poiseuille flow, 2-D pipe 0.16 x 0.02 m, 3200 x 300 cells, "
                "uniform inlet 0.01 sin(pi t) m/s, p = 0 outlet")
    if w["dim"] == 3:
        return f"{name}: 3-D lid-driven cavity {w['n']}^3 hex cells"
    return f"{name}: 2-D lid-driven cavity"


def cg_bytes_per_iter(N, F):
    """Algorithmic bytes of one Jacobi-PCG iteration (FP64 values, int32
    indices): SMVP + p.q reads diag, upper, owner/neighbour and p and writes
    q (24N + 16F); the r update with r.z reads q, r, 1/diag and writes r
    (32N); the x and p updates read x, p, r, 1/diag and write x, p (48N)."""
    return 104 * N + 16 * F


def cg_flops_per_iter(N, F):
    """Algorithmic FP64 flops of one Jacobi-PCG iteration: SMVP 2(N + 2F),
    p.q 2N, two axpys 4N, z = r/d N, r.z 2N, p update 2N, ||r||^2 2N."""
    return 15 * N + 4 * F


def fp64_peak_tflops(dev, sm_mhz):
    """FP64 peak from unit counts and clock: GB300 issues 2 FP64 FMA per
    clock per SM (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
    peak_sustained = 2 per cycle per SM)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return 2 * 2 * sms * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, fl in rows for k, v in enumerate(fl) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v, device):
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def source_sha1():
    """Hash of the CG kernel's source (the barrier and reductions of
    coop.cuh, k_pcg in krylov.cu): the recorded ncu traffic is reported only
    while this source is unchanged."""
    csrc = os.path.join(ROOT, "paper_1207_1571_gb300", "csrc")
    with open(os.path.join(csrc, "coop.cuh")) as f:
        coop = f.read()
    with open(os.path.join(csrc, "krylov.cu")) as f:
        src = f.read()
    a = src.index("// ------------------------------------------------------------------ CG --")
    b = src.index("// ------------------------------------------------------ mixed precision --")
    return hashlib.sha1((coop + src[a:b]).encode()).hexdigest()


# ------------------------------------------------------------------ ours --

# Algorithmic bytes of one launch of each assembly / correction stage (FP64
# values, int32 indices; each distinct array counted once per launch,
# neighbour gathers assumed to hit in cache).
def stage_bytes(N, F):
    return {
        # a1 momentum matrix (48F + 40N) and a2 Gauss gradient of p (16F + 32N)
        "momentum": 64 * F + 72 * N,
        # a4 H/A and rAU, a5 predicted flux, a6 pressure matrix (56F + 80N)
        "hbya+pressure": 56 * F + 80 * N,
        # a8 flux correction (reads phi*, a_f, writes phi: 24F, p 8N) and a9
        # Gauss gradient (16F + 32N) with u = HbyA - rAU grad p (56N)
        "correct": 40 * F + 96 * N,
    }


def mixed_kernel(resident=True):
    """The mixed-precision CG kernel the library runs: the Chronopoulos-Gear
    order where its row vectors fit in shared memory, the textbook order
    otherwise (FVGB_MIXED_CG forces one)."""
    form = os.environ.get("FVGB_MIXED_CG")
    if form == "classic" or (form != "cgcg" and not resident):
        return "k_pcg_mixed"
    return "k_pcg_mixed_cgcg"


def mixed_bytes_per_iter(N, F):
    """Algorithmic bytes of one FP32 inner iteration of the mixed-precision
    CG (FP32 values, int32 indices): product (12N + 12F), residual update
    (16N), direction and correction updates (24N)."""
    return 52 * N + 12 * F


def stage_rooflines(prof_ms, prof_n, N, F, peak, peak_kind):
    """Per-stage effective bandwidth from the stage timers of the timed steps
    (CUDA events around each launch on the library stream)."""
    names = {"momentum": [0], "hbya+pressure": [2, 3], "correct": [5]}
    sb = stage_bytes(N, F)
    out = {}
    for name, ks in names.items():
        ms = sum(prof_ms[k] for k in ks)
        n = prof_n[ks[-1]]          # launches of the pass (hbya and pressure pair up)
        if n <= 0 or ms <= 0:
            continue
        us = 1e3 * ms / n
        gbs = sb[name] / us / 1e3
        out[name] = {"us_per_launch": us, "bytes_per_launch": sb[name], "gbs": gbs,
                     "frac": gbs / peak, "peak_kind": peak_kind}
    return out


class StepTimer:
    """Times PISO steps of one case from rest: events on the library stream
    around every step, L2 flushed (256 MiB write) before each, stage timers
    on, statistics read after each step's end event."""

    def __init__(self, L, stream, flush):
        self.L, self.stream, self.flush = L, stream, flush

    def run(self, case, step, nsteps, stats=True):
        import torch
        import ctypes as C
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        self.L.fv_profile_read(None, None, 1)
        self.L.fv_profile_enable(1)
        its_p, its_u, per_solve, statuses, outer = 0, 0, [], [], 0
        torch.cuda.synchronize()
        for k in range(nsteps):
            with torch.cuda.stream(self.stream):
                self.flush.zero_()
                ev[k][0].record(self.stream)
            step(k, case.h)
            with torch.cuda.stream(self.stream):
                ev[k][1].record(self.stream)
            if stats:
                st = case.last_stats()
                its_p += sum(st["iters"][3:])
                its_u += sum(st["iters"][:3])
                per_solve.extend(int(x) for x in st["iters"][3:])
                statuses.append(st["status"])
                outer += sum(x["outer"] for x in st["p"])
        torch.cuda.synchronize()
        self.L.fv_profile_enable(0)
        ms = (C.c_double * 7)()
        n = (C.c_int64 * 7)()
        self.L.fv_profile_read(ms, n, 1)
        return {"t": sum(a.elapsed_time(b) for a, b in ev) / 1e3, "ms": list(ms), "n": list(n),
                "its_p": its_p, "its_u": its_u, "per_solve": per_solve,
                "statuses": statuses, "outer": outer}


def run_ours(args, ws, rank, local):
    import torch
    import ctypes as C
    from paper_1207_1571_gb300 import build as B
    import paper_1207_1571_gb300 as P
    from paper_1207_1571_gb300 import _capi

    if ws == 1:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    B.build()
    L = P.load()
    w = WORKLOADS[args.workload]
    m = make_mesh(w)
    N, F = m.n_cells, m.n_internal_faces
    mesh = P.Mesh(m, renumber=True)
    case = P.Case(mesh, w["nu"])
    ref = ref_cell(w, m)
    prm = case.piso_params(w["dt"], w["n_corr"], p_ref_cell=ref)
    stream = mesh.stream
    zero = (torch.zeros(3, N, dtype=torch.float64, device="cuda"),
            torch.zeros(N, dtype=torch.float64, device="cuda"),
            torch.zeros(m.n_faces, dtype=torch.float64, device="cuda"))
    st = _capi.fv_step_stats()

    def step(k, h, with_stats=False):
        set_bc(L, h, w, m, k)
        rc = L.fv_piso_step(h, C.byref(prm), C.byref(st) if with_stats else None)
        _capi.check(rc, "fv_piso_step", allow=(4,))
        return st

    def warm(c):
        for k in range(args.warmup):
            step(k, c.h)
        c.set_fields(*zero)
        torch.cuda.synchronize()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    timer = StepTimer(L, stream, flush)
    warm(case)
    barrier(ws)
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        r64 = timer.run(case, step, args.steps)
    barrier(ws)
    t_local = r64["t"]
    prof_ms, prof_n = r64["ms"], r64["n"]
    iters_p, iters_u, per_solve = r64["its_p"], r64["its_u"], r64["per_solve"]
    t = allmax(ws, t_local, "cuda")
    value = ws * N * args.steps / t
    pcg_s = prof_ms[4] / 1e3
    bpi = cg_bytes_per_iter(N, F)
    peak, peak_kind = peaks()
    achieved = bpi * iters_p / pcg_s / 1e9 if pcg_s > 0 else None
    traffic = None
    n_solves = max(1, len(per_solve))
    if (PCG_TRAFFIC["source_sha1"] == source_sha1() and PCG_TRAFFIC["bytes_per_iter"]
            and PCG_TRAFFIC["workload"] == args.workload):
        # per launch = per-iteration DRAM bytes x mean iterations per launch
        traffic = PCG_TRAFFIC["bytes_per_iter"] * iters_p / n_solves
    clk_sum = clk.summary()
    sm_mhz = clk_sum.get("sm_mhz") or 2070.0
    fp64_peak = fp64_peak_tflops(dev, sm_mhz)
    flops = cg_flops_per_iter(N, F) * iters_p
    fp64_achieved = flops / pcg_s / 1e12 if pcg_s > 0 else None
    # the CG's arrays of one iteration against the L2 size: at twice L2 or
    # less, most of an iteration's reads hit L2 (or the CG's own shared memory)
    l2_bytes = torch.cuda.get_device_properties(dev).L2_cache_size
    resident = bpi <= 2 * l2_bytes

    # the same steps with the mixed-precision pressure solve
    mixed = None
    if not args.no_mixed:
        cm = P.Case(mesh, w["nu"], P.FV_PREC_MIXED)
        warm(cm)
        rm = timer.run(cm, step, args.steps)
        tm = allmax(ws, rm["t"], "cuda")
        ua, pa, fa = case.get_fields()
        ub, pb_, fb = cm.get_fields()
        d_ = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        inner = rm["its_p"]
        mixed = {"value": ws * N * args.steps / tm, "unit": UNIT, "steps_per_s": args.steps / tm,
                 "speedup_vs_fp64": t / tm, "inner_iterations": inner, "outer_passes": rm["outer"],
                 "cg_ms": rm["ms"][4], "us_per_inner_iter": 1e3 * rm["ms"][4] / inner if inner else None,
                 "rel_l2_vs_fp64_gpu": {"u": d_(ub, ua), "p": d_(pb_, pa), "phi": d_(fb, fa),
                                        "p_meanfree": d_(pb_ - pb_.mean(), pa - pa.mean())}}
        if inner:
            mb = mixed_bytes_per_iter(N, F) * inner / (rm["ms"][4] / 1e3) / 1e9
            mixed["roofline"] = {"bound": "hbm", "kernel": mixed_kernel(resident), "achieved": mb,
                                 "peak": peak, "unit": "GB/s", "frac": mb / peak,
                                 "peak_kind": peak_kind,
                                 "algorithmic": "52N+12F bytes per FP32 inner iteration"}
        cm.close()

    formats = None if args.no_formats else spmv_formats(P, mesh, m, stream)
    table3 = None if args.no_formats else table3_ratios(P, mesh, m, stream, prof_ms, prof_n)

    # the same steps with the aggregation-multigrid preconditioned pressure CG
    amg = None
    if not args.no_amg:
        ca = P.Case(mesh, w["nu"])
        ca.set_pressure_solver(P.FV_PSOLVER_AMG)
        warm(ca)
        ra = timer.run(ca, step, args.steps)
        ta = allmax(ws, ra["t"], "cuda")
        ua, pa_, fa = case.get_fields()
        ub, pb_, fb = ca.get_fields()
        d_ = lambda x, y: float(torch.linalg.norm(x - y) / torch.linalg.norm(y))
        its_a = ra["its_p"]
        amg = {"value": ws * N * args.steps / ta, "unit": UNIT, "steps_per_s": args.steps / ta,
               "speedup_vs_jacobi_cg": t / ta, "levels": mesh.amg_levels(),
               "cg_iterations": its_a, "per_solve": ra["per_solve"], "cg_ms": ra["ms"][4],
               "us_per_iter": 1e3 * ra["ms"][4] / its_a if its_a else None,
               "rel_l2_vs_jacobi_cg": {"u": d_(ub, ua), "p": d_(pb_, pa_), "phi": d_(fb, fa),
                                       "p_meanfree": d_(pb_ - pb_.mean(), pa_ - pa_.mean())}}
        ca.close()
        # and with the V-cycle in FP32 (a mixed-precision case)
        cx = P.Case(mesh, w["nu"], P.FV_PREC_MIXED)
        cx.set_pressure_solver(P.FV_PSOLVER_AMG)
        warm(cx)
        rx = timer.run(cx, step, args.steps)
        tx = allmax(ws, rx["t"], "cuda")
        uc, pc, fc = cx.get_fields()
        amg["fp32_cycle"] = {"value": ws * N * args.steps / tx, "unit": UNIT,
                             "speedup_vs_jacobi_cg": t / tx, "cg_iterations": rx["its_p"],
                             "rel_l2_vs_fp64_cycle": {"u": d_(uc, ub), "p": d_(pc, pb_),
                                                      "phi": d_(fc, fb)}}
        cx.close()

    # end to end through the C ABI with host buffers
    e2e = None
    e2e_steps = args.steps if args.e2e_steps < 0 else args.e2e_steps
    if e2e_steps > 0:
        # the same steps as the device-timed value (from rest), the fields
        # in pinned host buffers, each step's inputs set from them and its
        # result read back into them
        case.set_fields(*zero)
        torch.cuda.synchronize()

        def pinned(*shape):
            return torch.zeros(shape, dtype=torch.float64, pin_memory=True).numpy()
        hu, hp, hphi = pinned(3, N), pinned(N), pinned(m.n_faces)
        te = 0.0
        for k in range(e2e_steps):
            t0 = time.perf_counter()
            _capi.check(L.fv_case_set_fields_host(case.h, hu.ctypes.data, hp.ctypes.data,
                                                  hphi.ctypes.data, 1), "set_fields_host")
            step(k, case.h)
            _capi.check(L.fv_case_get_fields_host(case.h, hu.ctypes.data, hp.ctypes.data,
                                                  hphi.ctypes.data, 1), "get_fields_host")
            te += time.perf_counter() - t0
        te = allmax(ws, te, "cuda")
        nbytes = 8 * (3 * N + N + m.n_faces)
        e2e = {"value": ws * N * e2e_steps / te, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": e2e_steps, "host_buffers": "pinned"}

    mem = case.memory_bytes()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "steps_per_s": args.steps / t,
        "config": {"workload": workload_name(args.workload, w, m),
                   "cells": N, "internal_faces": F, "nu": w["nu"], "dt": w["dt"],
                   "n_corr": w["n_corr"], "p_tol": 1e-6,
                   "renumbering": "RCM" if w.get("tp") or w.get("seed") is None
                   else f"seed-{w['seed']} permutation + RCM",
                   "l2": "flushed (256 MiB write) between timed steps; steps timed from rest",
                   "parallelism": "replicas only" if ws > 1 else "1 GPU"},
        "cg": {"iterations": iters_p, "iters_per_step": iters_p / args.steps,
               "per_solve": per_solve,
               "us_per_iter": 1e3 * prof_ms[4] / iters_p if iters_p else None,
               "bicgstab_iterations": iters_u, "ms": prof_ms[4],
               "share_of_step": prof_ms[4] / (1e3 * t_local) if t_local > 0 else None},
        "stages_ms": {n: prof_ms[k] for k, n in enumerate(_capi.PROF_STAGES)},
        "stage_rooflines": stage_rooflines(prof_ms, prof_n, N, F, peak, peak_kind),
        "roofline": {"bound": "hbm", "kernel": "k_pcg", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak if achieved else None,
                     "peak_kind": peak_kind, "traffic": traffic,
                     "bytes_per_iter": bpi, "algorithmic": "104N+16F bytes per CG iteration",
                     "note": ("effective bandwidth: the CG working set fits in L2 and shared "
                              "memory, so DRAM carries far less than the algorithmic bytes; the "
                              "FP64 pipe (roofline_fp64) is the binding limit here")
                     if resident else "working set larger than L2: HBM-bound"},
        "roofline_fp64": {"bound": "alu", "kernel": "k_pcg", "achieved": fp64_achieved,
                          "peak": fp64_peak, "unit": "TFLOP/s",
                          "frac": fp64_achieved / fp64_peak if fp64_achieved else None,
                          "peak_kind": "derived: 2 FP64 FMA/clk/SM x SMs x median SM clock x 2",
                          "algorithmic": "15N+4F flops per CG iteration"},
        "gpu_launches": int(sum(prof_n[k] for k in range(7))),
        "clocks": clk_sum,
        "e2e": e2e,
        "mixed": mixed,
        "spmv_formats": formats,
        "table3": table3,
        "amg": amg,
        "memory_bytes": mem,
        "bytes_per_cell": {"value": mem / N, "paper": 540,
                           "note": "device bytes of mesh + case (solver work space included) per "
                                   "cell; the paper's C2070 code needed about 540 (Sec. 4.3.4)"},
        "statuses": sorted(set(r64["statuses"])),
    }
    case.close()
    mixed_its = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, ofields = cpu_baseline(args.workload)
        out["cpu_baseline"] = cb
        # error of the first step from rest against the oracle's (FP64 and mixed)
        errs = {}
        for name, prec in (("fp64", P.FV_PREC_FP64), ("mixed", P.FV_PREC_MIXED)):
            c1 = P.Case(mesh, w["nu"], prec)
            step(0, c1.h)
            g = c1.get_fields_host()
            errs[name] = field_errors(g, ofields)
            c1.close()
        out["first_step_rel_l2_vs_oracle"] = errs
    mesh.close()
    if args.workload == "cavity3d_100" and ws == 1 and not args.no_extra_configs:
        del zero
        torch.cuda.empty_cache()
        out["cavity3d_200"] = run_c3(args, P, L, dev, peak, peak_kind)
        torch.cuda.empty_cache()
        out["batch256"] = {"fp64": run_batch(args, ws, rank, "fp64", line=False),
                           "mixed": run_batch(args, ws, rank, "mixed", line=False, loop=False)}
        out["batch256"]["mixed"]["speedup_vs_per_case_loop"] = (
            out["batch256"]["mixed"]["value"] / out["batch256"]["fp64"]["per_case_loop"]["value"])
    return out


def field_errors(got, ref):
    """Relative L2 error of each field, the pressure split into its mean-free
    part and its mean (relative to the RMS of the reference pressure)."""
    (u, p, phi), (uo, po, phio) = got, ref
    r = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    rms = float(np.sqrt(np.mean(po ** 2)))
    return {"u": r(u, uo), "p": r(p, po), "phi": r(phi, phio),
            "p_meanfree": r(p - p.mean(), po - po.mean()),
            "p_mean": abs(float(p.mean() - po.mean())) / (rms if rms > 0 else 1.0)}


def run_c3(args, P, L, dev, peak, peak_kind):
    """The 200^3 = 8M-cell cavity (nu 0.01, dt 0.001, 2 correctors), FP64
    and mixed-precision pressure solves, its stated 20 steps from rest after
    the same warm-up, timed like the main line."""
    import torch
    import ctypes as C
    from paper_1207_1571_gb300 import _capi
    name = "cavity3d_200"
    w = WORKLOADS[name]
    nsteps = 20
    m = make_mesh(w)
    N, F = m.n_cells, m.n_internal_faces
    mesh = P.Mesh(m, renumber=True)
    prm = P.Case.piso_params(w["dt"], w["n_corr"], p_ref_cell=m.corner_cell)

    def step(k, h):
        _capi.check(L.fv_piso_step(h, C.byref(prm), None), "fv_piso_step", allow=(4,))

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    timer = StepTimer(L, mesh.stream, flush)
    res = {"workload": workload_name(name, w, m), "cells": N, "internal_faces": F,
           "nu": w["nu"], "dt": w["dt"], "steps": nsteps, "warmup": args.warmup}
    fields = {}
    for prec_name, prec in (("fp64", P.FV_PREC_FP64), ("mixed", P.FV_PREC_MIXED)):
        c = P.Case(mesh, w["nu"], prec)
        for k in range(args.warmup):
            step(k, c.h)
        c.set_fields(torch.zeros(3, N, dtype=torch.float64, device="cuda"),
                     torch.zeros(N, dtype=torch.float64, device="cuda"),
                     torch.zeros(m.n_faces, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        with Clocks(dev) as clk:
            r = timer.run(c, step, nsteps)
        its, cg_s = r["its_p"], r["ms"][4] / 1e3
        d = {"value": N * nsteps / r["t"], "unit": UNIT, "steps_per_s": nsteps / r["t"],
             "ms_per_step": 1e3 * r["t"] / nsteps, "cg_iterations": its, "cg_ms": r["ms"][4],
             "us_per_iter": 1e6 * cg_s / its if its else None, "clocks": clk.summary(),
             "statuses": sorted(set(r["statuses"]))}
        bpi = cg_bytes_per_iter(N, F) if prec == P.FV_PREC_FP64 else mixed_bytes_per_iter(N, F)
        if its and cg_s > 0:
            gbs = bpi * its / cg_s / 1e9
            d["roofline"] = {"bound": "hbm",
                             "kernel": "k_pcg" if prec == P.FV_PREC_FP64 else mixed_kernel(False),
                             "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                             "peak_kind": peak_kind, "bytes_per_iter": bpi,
                             "algorithmic": "104N+16F bytes per CG iteration"
                             if prec == P.FV_PREC_FP64 else "52N+12F bytes per FP32 inner iteration"}
        if prec == P.FV_PREC_FP64:
            d["stage_rooflines"] = stage_rooflines(r["ms"], r["n"], N, F, peak, peak_kind)
        else:
            d["outer_passes"] = r["outer"]
        fields[prec_name] = c.get_fields_host()
        res[prec_name] = d
        c.close()
    res["mixed"]["speedup_vs_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    res["mixed"]["rel_l2_vs_fp64_gpu"] = field_errors(fields["mixed"], fields["fp64"])
    mesh.close()
    return res


def table3_ratios(P, mesh, m, stream, prof_ms, prof_n, reps=20):
    """The paper's Table 3 compares the time of its assembly operators with
    one SMVP (Sec. 4.3.3).  Here: one LDU product through the SELL rows
    (fv_ldu_matvec), one Gauss gradient (fv_gauss_grad), and per launch of the
    fused kernels of the timed steps -- the pressure assembly (divergence of
    the predicted flux plus the Laplacian's coefficients) and the momentum
    assembly (convection, diffusion Laplacian and grad p)."""
    import torch
    N, F = m.n_cells, m.n_internal_faces
    g = torch.Generator(device="cuda").manual_seed(5)
    d = torch.rand(N, dtype=torch.float64, device="cuda", generator=g) + 4
    up = torch.randn(F, dtype=torch.float64, device="cuda", generator=g)
    x = torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
    xb = torch.randn(m.n_boundary_faces, dtype=torch.float64, device="cuda", generator=g)
    L = mesh.L
    y = torch.empty_like(x)
    gr = torch.empty(3, N, dtype=torch.float64, device="cuda")
    ops = {"smvp": lambda: L.fv_ldu_matvec(mesh.h, d.data_ptr(), up.data_ptr(), up.data_ptr(),
                                            x.data_ptr(), y.data_ptr()),
           "grad": lambda: L.fv_gauss_grad(mesh.h, x.data_ptr(), xb.data_ptr(), gr.data_ptr())}
    us = {}
    torch.cuda.synchronize()
    for name, fn in ops.items():
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            rc = fn()
            if rc != 0:
                raise RuntimeError(f"{name} failed with status {rc}")
        b.record(stream)
        b.synchronize()
        us[name] = 1e3 * a.elapsed_time(b) / reps
    per = lambda k: 1e3 * prof_ms[k] / prof_n[k] if prof_n[k] else None
    pres, mom = per(3), per(0)
    return {"smvp_us": us["smvp"], "grad_us": us["grad"], "pressure_assembly_us": pres,
            "momentum_assembly_us": mom,
            "grad_over_smvp": us["grad"] / us["smvp"],
            "div_plus_laplacian_over_smvp": pres / us["smvp"] if pres else None,
            "momentum_assembly_over_smvp": mom / us["smvp"] if mom else None,
            "paper_c2070": {"div_over_smvp": "2.5-4.1", "grad_over_smvp": "9.0-18.3",
                            "laplacian_over_smvp": "2.3-2.5 (58.7 on the non-orthogonal lca mesh)"}}


def spmv_formats(P, mesh, m, stream, reps=20):
    """One matrix-vector product in each storage, on the workload's mesh:
    the LDU face arrays read through the SELL-32 rows (fv_ldu_matvec), and
    the paper's hybrid ELL + J storage by rows (SMVP) and by columns
    (STMVP, through I and J or the packed Q).  Mean device time of `reps`
    products after one warm-up, CUDA events on the library stream; GB/s
    from the arrays each product reads and writes once."""
    import torch
    N, F = m.n_cells, m.n_internal_faces
    g = torch.Generator(device="cuda").manual_seed(3)
    d = torch.rand(N, dtype=torch.float64, device="cuda", generator=g) + 4
    up = torch.randn(F, dtype=torch.float64, device="cuda", generator=g)
    lo = torch.randn(F, dtype=torch.float64, device="cuda", generator=g)
    x = torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
    y = torch.empty_like(x)
    e = P.Ellj(mesh)
    V, Cv = e.from_ldu(d, up, lo)
    L = mesh.L
    nnz = N + 2 * F
    K = e.K
    ops = {
        "ldu_sell32": (lambda: L.fv_ldu_matvec(mesh.h, d.data_ptr(), up.data_ptr(), lo.data_ptr(),
                                               x.data_ptr(), y.data_ptr()),
                       8 * N + 16 * F + 8 * 2 * F + 16 * N),
        "ellj_smvp": (lambda: L.fv_ellj_spmv(e.h, V.data_ptr(), Cv.data_ptr(), x.data_ptr(),
                                             y.data_ptr(), 0), 12 * K * N + 16 * N),
        "ellj_stmvp": (lambda: L.fv_ellj_spmv(e.h, V.data_ptr(), Cv.data_ptr(), x.data_ptr(),
                                              y.data_ptr(), 1), 16 * K * N + 16 * N),
    }
    if e.n_crs == 0:
        ops["ellj_stmvp_q"] = (lambda: L.fv_ellj_spmv(e.h, V.data_ptr(), Cv.data_ptr(), x.data_ptr(),
                                                      y.data_ptr(), 2), 12 * K * N + 16 * N)
    out = {"K": K, "n_crs": e.n_crs, "nnz": nnz}
    torch.cuda.synchronize()
    for name, (fn, nbytes) in ops.items():
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            rc = fn()
            if rc != 0:
                raise RuntimeError(f"{name} failed with status {rc}")
        b.record(stream)
        b.synchronize()
        us = 1e3 * a.elapsed_time(b) / reps
        out[name] = {"us": us, "gbs": nbytes / us / 1e3, "bytes": nbytes}
    e.close()
    return out


def host_cpu():
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def cpu_baseline(workload):
    """The oracle as it stands, one PISO step of the same workload from rest
    (the first step of the timed sequence): its OpenMP build on all host
    cores (the reported baseline; fixed-block sums, results independent of
    the thread count) and its sequential build on one core."""
    import oracle as O
    w = WORKLOADS[workload]
    m = make_mesh(w)
    res = {}
    fields = None
    for par in (True, False):
        if par:
            O.set_threads(os.cpu_count() or 1)
        om = O.Mesh(m, renumber=True, parallel=par)
        oc = O.Case(om, w["nu"])
        t0 = time.perf_counter()
        if w.get("tp"):
            import meshgen as mg
            oc.set_patch(m.patch("inlet"), mg.tp_inlet(w["dt"]), 0.0)
        oc.piso_step(w["dt"], w["n_corr"], p_ref_cell=ref_cell(w, m))
        res[par] = time.perf_counter() - t0
        if par:
            fields = oc.get_fields()
        del oc, om
    nt = O.threads()
    cpu = host_cpu()
    cb = {"value": m.n_cells / res[True], "unit": UNIT, "cores": nt, "kind": "oracle",
          "sample": f"1 PISO step from rest of {workload} ({m.n_cells} cells), FP64 C oracle, "
                    f"OpenMP build on {nt} threads of {cpu['nproc']} ({cpu['model']}), "
                    f"{res[True]:.1f} s",
          "single_thread": {"value": m.n_cells / res[False], "unit": UNIT, "cores": 1,
                            "sample": f"the same step, sequential build, {res[False]:.1f} s"},
          "host": cpu}
    return cb, fields


# ----------------------------------------------------------------- batch --

def run_batch(args, ws, rank, precision=None, line=True, loop=True):
    """256 independent 2-D cavities (n ~ U[32,128], Re log-uniform in
    [10,1000], seed 7): batched steps (one launch per PISO stage, CUDA graph,
    autotuned schedule) against a per-case loop of the single-case solver
    over the same number of steps from rest."""
    import torch
    import ctypes as C
    import meshgen as mg
    from paper_1207_1571_gb300 import build as B
    import paper_1207_1571_gb300 as P
    from paper_1207_1571_gb300 import _capi
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    L = P.load()
    precision = precision or args.precision
    spec = mg.batch_cases(BATCH["n_cases"], BATCH["seed"])
    ms = [mg.cavity2d(n) for n, _ in spec]
    nus = [nu for _, nu in spec]
    refs = [m.corner_cell for m in ms]
    ncell = sum(m.n_cells for m in ms)
    nface = sum(m.n_internal_faces for m in ms)
    dt, nc = BATCH["dt"], BATCH["n_corr"]
    prec = P.FV_PREC_MIXED if precision == "mixed" else P.FV_PREC_FP64
    warm = P.Batch(ms, nus, refs, prec)
    key = f"{torch.cuda.get_device_name()}|batch{len(ms)}|seed{BATCH['seed']}|{precision}"
    if args.schedule is not None:
        warm.set_schedule(args.schedule)
        tuned = dict(schedule=args.schedule, given=True, **P.Batch.schedules()[args.schedule])
    else:
        tuned = warm.autotune(dt, nc, cache_path=os.path.join(ROOT, "paper_1207_1571_gb300",
                                                               "_build", "autotune.json"), key=key)
    for _ in range(args.warmup):
        warm.run_graph(1, dt, nc, stats=False)
    torch.cuda.synchronize()
    warm.close()
    bt = P.Batch(ms, nus, refs, prec, stream=torch.cuda.Stream())
    bt.set_schedule(tuned["schedule"])
    prm = P.Case.piso_params(dt, nc)
    stream = bt.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # capture once outside the timed region
    _capi.check(L.fv_batch_run_graph(bt.h, C.byref(prm), 0, None), "fv_batch_run_graph")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[k][0].record(stream)
            _capi.check(L.fv_batch_run_graph(bt.h, C.byref(prm), 1, None), "fv_batch_run_graph")
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    t = allmax(ws, sum(a.elapsed_time(b) for a, b in ev) / 1e3, "cuda")
    # two more steps launched directly with the stage timers and statistics:
    # CG share of a step and iterations per case for the roofline
    L.fv_profile_read(None, None, 1)
    L.fv_profile_enable(1)
    its = np.zeros(len(ms))
    for _ in range(2):
        st = bt.piso_step(dt, nc)
        its += [sum(s["iters"][3:]) for s in st]
    torch.cuda.synchronize()
    L.fv_profile_enable(0)
    pm = (C.c_double * 7)()
    pn = (C.c_int64 * 7)()
    L.fv_profile_read(pm, pn, 1)
    peak, peak_kind = peaks()
    if prec == P.FV_PREC_FP64:
        bytes_cg = sum(cg_bytes_per_iter(mm.n_cells, mm.n_internal_faces) * k for mm, k in zip(ms, its))
        kern, alg = "k_pcg_batch", "sum over cases of (104N+16F) x CG iterations"
    else:
        bytes_cg = sum(mixed_bytes_per_iter(mm.n_cells, mm.n_internal_faces) * k for mm, k in zip(ms, its))
        kern, alg = "k_pcg_mixed_batch", "sum over cases of (52N+12F) x FP32 inner iterations"
    gbs = bytes_cg / (pm[4] / 1e3) / 1e9 if pm[4] > 0 else None
    roof = {"bound": "hbm", "kernel": kern, "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak if gbs else None, "peak_kind": peak_kind, "algorithmic": alg,
            "cg_share_of_direct_steps": pm[4] / sum(pm[k] for k in range(7)) if pm[4] else None,
            "direct_steps_stage_ms": {n: pm[k] / 2 for k, n in enumerate(_capi.PROF_STAGES)}}
    value = ws * ncell * args.steps / t
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec == P.FV_PREC_FP64 else "f64+f32", "data": "synthetic",
           "steps_per_s": args.steps / t,
           "config": {"workload": "batch256: 256 independent 2-D lid-driven cavities, n_i in "
                                  "[32,128], Re_i log-uniform in [10,1000] (seed 7), dt 0.002, "
                                  "PISO 2 correctors", "cells": ncell, "internal_faces": nface,
                      "cases": len(ms), "schedule": tuned,
                      "l2": "flushed between timed steps; steps from rest",
                      "precision": precision},
           "cg_iterations_per_step": float(its.sum() / 2), "roofline": roof,
           "clocks": clk.summary(), "gpu_launches": 10 * args.steps}
    bt.close()
    if loop:
        # per-case loop of the single-case solver: the same cases from rest,
        # the same number of steps
        meshes = [P.Mesh(m, renumber=True, stream=stream) for m in ms]
        cases = [P.Case(mm, nu) for mm, nu in zip(meshes, nus)]
        prms = [P.Case.piso_params(dt, nc, p_ref_cell=r) for r in refs]
        for c, pr in zip(cases, prms):
            L.fv_piso_step(c.h, C.byref(pr), None)
        torch.cuda.synchronize()
        for c in cases:
            c.set_fields(torch.zeros(3, c.mesh.N, dtype=torch.float64, device="cuda"),
                         torch.zeros(c.mesh.N, dtype=torch.float64, device="cuda"),
                         torch.zeros(c.mesh.M, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for c, pr in zip(cases, prms):
                _capi.check(L.fv_piso_step(c.h, C.byref(pr), None), "fv_piso_step")
        e1.record(stream)
        torch.cuda.synchronize()
        t_loop = e0.elapsed_time(e1) / 1e3
        v_loop = ncell * args.steps / t_loop
        out["per_case_loop"] = {"value": v_loop, "unit": UNIT, "steps": args.steps,
                                "ms_per_step": 1e3 * t_loop / args.steps}
        out["speedup_vs_per_case_loop"] = value / ws / v_loop
        for c in cases:
            c.close()
        for mm in meshes:
            mm.close()
    if not line:
        for k in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data"):
            out.pop(k, None)
    return out


# ------------------------------------------------------------- reference --

def run_reference(args, ws, rank):
    """The reference arm: the FP64 CPU oracle (OpenMP build, all host cores)
    on the workload's own mesh, the first REF_STEPS PISO steps from rest."""
    if rank != 0:
        return None
    import oracle as O
    w = WORKLOADS[args.workload]
    if w.get("batch"):
        return {"impl": "reference", "unavailable": "the reference arm times single-case workloads"}
    m = make_mesh(w)
    O.set_threads(os.cpu_count() or 1)
    om = O.Mesh(m, renumber=True, parallel=True)
    oc = O.Case(om, w["nu"])
    nsteps = REF_STEPS
    t0 = time.perf_counter()
    for k in range(nsteps):
        if w.get("tp"):
            import meshgen as mg
            oc.set_patch(m.patch("inlet"), mg.tp_inlet((k + 1) * w["dt"]), 0.0)
        oc.piso_step(w["dt"], w["n_corr"], p_ref_cell=ref_cell(w, m))
    t = time.perf_counter() - t0
    v = m.n_cells * nsteps / t
    nt = O.threads()
    cpu = host_cpu()
    sample = (f"the first {nsteps} PISO steps from rest of {args.workload} itself "
              f"({m.n_cells} cells; --steps/--warmup not used: a bounded sample), FP64 C oracle, "
              f"OpenMP build on {nt} threads ({cpu['model']})")
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": nsteps,
            "warmup": 0, "ms_per_step": 1e3 * t / nsteps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(args.workload, w, m), "cells": m.n_cells,
                       "same_config": True},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cavity3d_100")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="end-to-end steps through host buffers (default: the same as --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-amg", action="store_true",
                    help="skip the multigrid-preconditioned pressure CG leg")
    ap.add_argument("--no-formats", action="store_true",
                    help="skip the SpMV storage comparison (SELL-32 vs ELL + J) and Table 3")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the 200^3 cavity and batch legs of the default run")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="batch workload only")
    ap.add_argument("--schedule", type=int, default=None,
                    help="batch workload only: fixed schedule instead of the autotuner")
    args = ap.parse_args()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    elif WORKLOADS[args.workload].get("batch"):
        out = run_batch(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
