#!/usr/bin/env python
"""Benchmark of the even-odd clover-Wilson hot path on GB300.

One step = one reliable-update mixed-precision CG solve of
(Mhat^dag Mhat) x = b to a TRUE FP64 residual <= 1e-10 |b| on a 32^3x64
lattice (kappa 0.1355, c_SW 1.9, links exp(i 0.15 A) reunitarised, antiperiodic
t), with the inner Krylov iteration in FP32 (12-real links) and FP64 residual
recomputation: every row of the hot path (hopping term, clover and inverse
epilogues, Mhat, Mhat^dag Mhat, BLAS-1 and reductions, FP64 CG outer updates)
runs inside it.

value = algorithmic hopping-term bytes of all launches in the timed solves
(8 links + in + out spinor per site, plus the clover blocks / x spinor the
fused epilogues read) / the timed wall time on the device, in GB/s. The line
also carries the plain FP64 CG time on the same system (the mixed/FP64
speed-up), the same solve with an FP16 inner iteration, a Dslash bandwidth
sweep per precision, the roofline of the dominant kernel, the CPU oracle
baseline, the end-to-end figure through the C ABI with host buffers, and the
batched and next-row measurements (12 point sources, 10-shift and block
multishift, ragged lattices, full-lattice BiCGstab / CG, trace samples, stout
step, clover log det), each against the same work done one system at a time
where that comparison exists. --mode selects another timed step.

--impl reference times the FP64 CPU oracle (the only reference there is: the
paper ships no code) on the same lattice, one Mhat^dag Mhat apply per step.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
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

METRIC = "Dslash GB/s vs HBM peak; mixed/batched vs FP64 CG time to |r|/|b|<1e-10"

WORKLOADS = {
    "48^3x96": dict(dims=(48, 48, 48, 96), eps=0.15, kappa=0.1355, csw=1.9, mu=0.0, seed=5, u1_sigma=0.1,
                    charges=(2.0 / 3.0, -1.0 / 3.0)),
    "32^3x64": dict(dims=(32, 32, 32, 64), eps=0.15, kappa=0.1355, csw=1.9, mu=0.0, seed=1),
    "24^3x48": dict(dims=(24, 24, 24, 48), eps=0.2, kappa=0.1350, csw=1.7, mu=0.0, seed=1),
    "20^3x40": dict(dims=(20, 20, 20, 40), eps=0.2, kappa=0.1350, csw=1.7, mu=0.0, seed=1),
    "16^3x32": dict(dims=(16, 16, 16, 32), eps=0.2, kappa=0.1350, csw=1.7, mu=0.0, seed=1),
    "8^4": dict(dims=(8, 8, 8, 8), eps=0.3, kappa=0.125, csw=1.0, mu=0.0, seed=1),
}
PREC_ID = {"double": 0, "single": 1, "half": 2}
SPINOR_B = {0: 192, 1: 96, 2: 52}
CLOVER_B = {0: 576, 1: 288, 2: 144}
EPI_NAMES = ["dhop", "dhop_clovinv", "dhop_xpay", "cg_mhat_norms", "cg_mhatdag_update"]


def link_b(prec, recon):
    return recon * {0: 8, 1: 4, 2: 2}[prec]


def mdagm_bytes(prec, recon, Vh):
    """Algorithmic bytes of one Mhat^dag Mhat: 2 D_oe+A^-1 and 2 A x - k D_eo launches."""
    clovinv = 8 * link_b(prec, recon) + 2 * SPINOR_B[prec] + CLOVER_B[prec]
    xpay = clovinv + SPINOR_B[prec]
    return 2.0 * (clovinv + xpay) * Vh


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="32^3x64", choices=sorted(WORKLOADS))
    ap.add_argument("--inner", default="single", choices=["single", "half", "double"],
                    help="precision of the inner Krylov iteration (double = plain FP64 CG)")
    ap.add_argument("--delta", type=float, default=None, help="reliable-update threshold (default 1e-3)")
    ap.add_argument("--check-every", type=int, default=8, help="iterations between host residual checks")
    ap.add_argument("--fp64-arith", default="df64", choices=["native", "df64"],
                    help="arithmetic of the FP64-storage operator kernels")
    ap.add_argument("--no-extras", action="store_true", help="skip FP64 CG, sweep, e2e and CPU baseline")
    ap.add_argument("--batch-mapping", type=int, default=0,
                    help="right-hand-side mapping of the batched modes (0 = autotuned; see bq_set_batch_mapping)")
    ap.add_argument("--mode", default="cg", choices=["cg", "batch12", "multishift10", "ragged4", "qed2x4",
                                                     "blockms4x10", "full_cg", "traces8"],
                    help="the timed step: one mixed CG solve (default), 12 point sources in one batched "
                         "solve, a 10-shift multishift solve, a ragged batch of four lattices, (48^3x96) "
                         "4 Gaussian sources for each of the two QED flavours in one batched solve, a block "
                         "multishift solve of 4 sources x 10 shifts, one full-lattice M x = b solve (CG on "
                         "Mhat^dag Mhat), or the trace samples of 8 Z2 noise vectors")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.idx = device_index
        try:
            cmd = ["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if device_index is not None:
                cmd += ["-i", str(device_index)]
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ traffic from the committed ncu summary

KERNEL_SOURCES = ("bq_device.cuh", "bq_stencil.cuh", "bq_cgfuse.cuh", "bq_cgfuse.cu")  # the files that define k_dslash, k_dslash_cg


def kernel_source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1711_03836_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel_tag, workload):
    """bytes per launch from a 'bench-traffic:' line of profiles/*.md, if the kernels are unchanged."""
    src = kernel_source_hash()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as f:
            for line in f:
                if line.startswith("bench-traffic:"):
                    parts = dict(kv.split("=", 1) for kv in line.split()[1:] if "=" in kv)
                    if (parts.get("kernel") == kernel_tag and parts.get("workload") == workload
                            and parts.get("src") == src):
                        return float(parts["bytes_per_launch"])
    return None


# ------------------------------------------------------------------ reference arm: the FP64 CPU oracle

def oracle_setup(wl):
    import oracle
    from paper_1711_03836_gb300 import synth

    U = synth.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    A = synth.u1_field(wl["dims"], wl["u1_sigma"], wl["seed"] + 1) if "u1_sigma" in wl else None
    charge = wl.get("charges", (0.0,))[0]
    p = oracle.params(wl["dims"], kappa=wl["kappa"], csw=wl["csw"], mu=wl["mu"], t_bc=-1.0, charge=charge)
    op = oracle.Operator(p, U, A)
    Vh = oracle.half_volume(p)
    b = synth.gaussian_spinor(Vh, wl["seed"] + 1000)
    return op, b, Vh


def oracle_gbs(op, b, Vh, steps, warmup, median=False):
    """(GB/s, seconds) of the oracle's Mhat^dag Mhat: the mean over `steps` applies, or their median."""
    for _ in range(warmup):
        op.mdagm(b)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        op.mdagm(b)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts) if median else sum(ts) / steps
    return mdagm_bytes(0, 18, Vh) / t / 1e9, t


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    wl = WORKLOADS[args.workload]
    op, b, Vh = oracle_setup(wl)
    gbs, t_step = oracle_gbs(op, b, Vh, args.steps, max(args.warmup, 0))
    cores = oracle.num_threads()
    sample = f"one FP64 Mhat^dag Mhat apply per step on the full {args.workload} lattice (no solve)"
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "lattice": list(wl["dims"])},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_name(args):
    wl = WORKLOADS[args.workload]
    d = "x".join(str(x) for x in wl["dims"])
    qed = (f" times U(1) phases exp(-i Q A_mu), sigma_A {wl['u1_sigma']}, Q in {list(wl['charges'])}"
           if "u1_sigma" in wl else "")
    return (f"{args.workload} ({d}) even-odd clover-Wilson, kappa {wl['kappa']}, c_SW {wl['csw']}, "
            f"links exp(i {wl['eps']} A) reunitarised{qed}, antiperiodic t; mixed-precision CG "
            f"({args.inner} inner, {'18' if 'u1_sigma' in wl else '12'}-real links, FP64-storage reliable updates "
            f"in {args.fp64_arith} arithmetic) "
            f"to true residual 1e-10")


# ------------------------------------------------------------------ our arm

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_1711_03836_gb300 import bqcd, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = WORKLOADS[args.workload]
    dims = wl["dims"]
    U = synth.gauge_field(dims, wl["eps"], wl["seed"])
    A = synth.u1_field(dims, wl["u1_sigma"], wl["seed"] + 1) if "u1_sigma" in wl else None
    charges = wl.get("charges", (0.0,))
    lat = bqcd.Lattice(dims, wl["kappa"], wl["csw"], wl["mu"], -1.0, charges[0])
    ctx = lat.ctx
    bqcd.bq_set_gauge(ctx, U)
    if A is not None:
        bqcd.bq_set_u1(ctx, A)
    else:
        bqcd.bq_set_recon(ctx, "single", 12)
        bqcd.bq_set_recon(ctx, "half", 12)
    field_inputs = (U, A)
    bqcd.bq_set_fp64_arith(ctx, args.fp64_arith)
    bqcd.bq_build_clover(ctx)
    Vh = lat.Vh
    b = synth.gaussian_spinor(Vh, wl["seed"] + 1000 + rank)
    b_dev = torch.from_numpy(b).cuda()
    x_dev = torch.empty_like(b_dev)
    delta = args.delta if args.delta is not None else {"single": 1e-3, "half": 1e-3, "double": 0.0}[args.inner]
    solve_kw = dict(tol=1e-10, precision=args.inner, delta=delta, check_every=args.check_every, max_iter=20000)

    bqcd.bq_set_batch_mapping(ctx, args.batch_mapping)
    step, extra_ctxs = make_step(args, torch, bqcd, synth, lat, b_dev, x_dev, solve_kw, field_inputs)
    del field_inputs, U, A
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K solves, inputs resident in HBM (launch counters on, no per-launch events)
    sampler = ClockSampler(None if world == 1 else local)
    barrier()
    torch.cuda.synchronize()
    bqcd.bq_reset_counters(ctx, timing=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record()
    for _ in range(args.steps):
        stats.append(step())
    e1.record()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    cnt_value = bqcd.bq_get_counters(ctx)
    total_bytes = sum(sum(r) for r in cnt_value["dslash_bytes"])
    # ---- second timed region, same K solves, with CUDA events around every hopping-term launch
    # (they cost a few microseconds per launch, so the value above is timed without them)
    bqcd.bq_reset_counters(ctx, timing=True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    cnt = bqcd.bq_get_counters(ctx)
    ms_max, bytes_all = aggregate_ranks(ms, total_bytes, "cuda") if world > 1 else (ms, total_bytes)
    value = bytes_all / (ms_max * 1e-3) / 1e9

    # dominant hopping-term kernel over the timed region (CUDA events around each launch)
    best = max(((p, e) for p in range(3) for e in range(5)), key=lambda pe: cnt["dslash_ms"][pe[0]][pe[1]])
    bp, be = best
    n_l = cnt["dslash_launches"][bp][be]
    # the CG-fused launches also move the vectors of the fused x / r update
    per_launch_bytes = (cnt["dslash_bytes"][bp][be] + cnt["fused_bytes"][bp][be]) / max(n_l, 1)
    per_launch_ms = cnt["dslash_ms"][bp][be] / max(n_l, 1)
    peak, peak_kind = measured_peaks()
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    tag = f"{'k_dslash_cg' if be >= 3 else 'k_dslash'}<{['double', 'single', 'half'][bp]},{EPI_NAMES[be]}>"
    traffic = committed_traffic(tag, args.workload)
    all_ms = sum(sum(r) for r in cnt["dslash_ms"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": tag, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": per_launch_bytes, "launches": n_l,
                "avg_launch_us": per_launch_ms * 1e3, "share_of_dslash_time": cnt["dslash_ms"][bp][be] / all_ms,
                "timing": "CUDA events around each launch, second timed pass of the same K steps"}
    # every hopping-term bucket of the solve: launches, mean CUDA-event time, algorithmic GB/s
    buckets = {}
    for p in range(3):
        for e in range(5):
            n = cnt["dslash_launches"][p][e]
            if n and cnt["dslash_ms"][p][e] > 0:
                us = cnt["dslash_ms"][p][e] / n * 1e3
                nbytes = (cnt["dslash_bytes"][p][e] + cnt["fused_bytes"][p][e]) / n
                buckets[f"{'k_dslash_cg' if e >= 3 else 'k_dslash'}<{['double', 'single', 'half'][p]},{EPI_NAMES[e]}>"] = {
                    "launches": n, "avg_us": us, "GB/s": nbytes / (us * 1e-6) / 1e9}
    roofline["buckets"] = buckets

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"single": "f32+f64", "half": "f16-storage/f32+f64", "double": "f64"}[args.inner],
        "data": "synthetic",
        "config": {"workload": workload_name(args), "lattice": list(dims), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (FP32 links 0.4 GB + clover 1.2 GB + FP64 links 1.2 GB)"},
        "roofline": roofline,
        "gpu_launches": cnt_value["launches"],
        "clocks": clocks,
        "solve": summarize(stats[-1]),
    }
    if args.mode != "cg":
        line["config"]["batch_mapping"] = bqcd.bq_get_batch_mapping(ctx)
    if args.mode != "cg":
        line["config"]["workload"] = f"{args.mode} on " + line["config"]["workload"]

    for l in extra_ctxs:
        l.close()
    if not args.no_extras and world == 1 and args.mode == "cg":
        line.update(extras(args, ctx, lat, b, b_dev, x_dev, solve_kw, ms_max / args.steps, torch, bqcd))
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


FP64_NOMINAL_GFLOPS = 1250.0


def measured_fp64_peak():
    """Sustained FP64 FMA rate of this GPU (GFLOP/s) from the DFMA-chain probe
    (paper_1711_03836_gb300/probe/bq_probe.cu), or the nominal 1.25 TFLOP/s."""
    import ctypes

    from paper_1711_03836_gb300 import build as cuda_build

    try:
        lib = ctypes.CDLL(cuda_build.build_probe())
        v = ctypes.c_double()
        if lib.bq_probe_dfma_gflops(5, ctypes.byref(v)) == 0 and v.value > 0:
            return v.value, "measured (DFMA-chain probe, best of 5 launches)"
    except Exception as e:  # the probe is a measurement aid; the bench still runs without it
        return FP64_NOMINAL_GFLOPS, f"nominal (probe failed: {e})"
    return FP64_NOMINAL_GFLOPS, "nominal (probe failed)"


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _timed(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, (time.perf_counter() - t0) * 1e3


def batched_extras(torch, bqcd, fp64_arith):
    """12 point sources and 10 RHMC shifts on 24^3x48, and a ragged set of four
    lattices: one batched solve against the same systems solved one at a time
    (mixed precision, FP32 inner, to a true FP64 residual 1e-10)."""
    from paper_1711_03836_gb300 import synth

    out = {}
    kw = dict(tol=1e-10, precision="single", delta=1e-3, check_every=8, max_iter=20000)
    wl = WORKLOADS["24^3x48"]
    lat = bqcd.Lattice(wl["dims"], wl["kappa"], wl["csw"], wl["mu"], -1.0)
    bqcd.bq_set_gauge(lat.ctx, synth.gauge_field(wl["dims"], wl["eps"], wl["seed"]))
    bqcd.bq_set_recon(lat.ctx, "single", 12)
    bqcd.bq_set_fp64_arith(lat.ctx, fp64_arith)
    srcs = [torch.from_numpy(synth.point_source(lat.Vh, 0, s, c)).cuda() for s in range(4) for c in range(3)]
    xs = [torch.empty_like(b) for b in srcs]
    bqcd.bq_solve_cg_batch([lat.ctx] * 12, xs, srcs, **kw)  # warm
    st_b, ms_b = _timed(torch, lambda: bqcd.bq_solve_cg_batch([lat.ctx] * 12, xs, srcs, **kw))
    mapping_b = bqcd.bq_get_batch_mapping(lat.ctx)
    st_s, ms_s = _timed(torch, lambda: [bqcd.bq_solve_cg(lat.ctx, x, b, **kw) for x, b in zip(xs, srcs)])
    out["point_sources_12_24^3x48"] = {
        "batched_ms": ms_b, "sequential_ms": ms_s, "speedup": ms_s / ms_b,
        "max_true_residual": max(s_["true_residual"] for s_ in st_b),
        "iterations_max": max(s_["iterations"] for s_ in st_b), "mapping": mapping_b}
    out["batched_apply_12_24^3x48"] = batched_apply_roofline(torch, bqcd, lat)
    # RHMC multishift: 10 shifts geometric over [1e-4, 1] vs 10 separate CG solves
    b = torch.from_numpy(synth.gaussian_spinor(lat.Vh, 77)).cuda()
    shifts = [10.0 ** (-4 + 4 * k / 9) for k in range(10)]
    xk = [torch.empty_like(b) for _ in shifts]
    bqcd.bq_solve_multishift_cg(lat.ctx, xk, b, shifts, tol=1e-10, precision="single", delta=1e-3)
    st_m, ms_m = _timed(torch, lambda: bqcd.bq_solve_multishift_cg(lat.ctx, xk, b, shifts, tol=1e-10,
                                                                     precision="single", delta=1e-3))
    st_10, ms_10 = _timed(torch, lambda: [bqcd.bq_solve_cg(lat.ctx, x, b, shift=sh, **kw)
                                          for x, sh in zip(xk, shifts)])
    out["multishift_10_24^3x48"] = {"multishift_ms": ms_m, "separate_cg_ms": ms_10, "speedup": ms_10 / ms_m,
                                    "worst_true_residual": st_m["true_residual"]}
    # block multishift: 4 right-hand sides x the same 10 shifts vs 4 multishift solves in turn
    b4 = [torch.from_numpy(synth.gaussian_spinor(lat.Vh, 780 + r)).cuda() for r in range(4)]
    x4 = [[torch.empty_like(b) for _ in shifts] for _ in b4]
    mkw = dict(tol=1e-10, precision="single", delta=1e-3)
    bqcd.bq_solve_multishift_cg_block(lat.ctx, x4, b4, shifts, **mkw)
    st_bm, ms_bm = _timed(torch, lambda: bqcd.bq_solve_multishift_cg_block(lat.ctx, x4, b4, shifts, **mkw))
    st_sm, ms_sm = _timed(torch, lambda: [bqcd.bq_solve_multishift_cg(lat.ctx, x4[r], b4[r], shifts, **mkw)
                                          for r in range(4)])
    out["block_multishift_4x10_24^3x48"] = {
        "block_ms": ms_bm, "multishift_in_turn_ms": ms_sm, "speedup": ms_sm / ms_bm,
        "worst_true_residual": max(s_["true_residual"] for s_ in st_bm),
        "krylov_plus_refinement_iterations_max": max(s_["iterations"] for s_ in st_bm)}
    del x4, b4
    lat.close()
    # ragged: 8^4, 12^4, 16^3x32, 20^3x40 in one batched solve
    lats, bs, xr = [], [], []
    for i, dims in enumerate([(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (20, 20, 20, 40)]):
        l = bqcd.Lattice(dims, 0.1350, 1.7, 0.0, -1.0)
        bqcd.bq_set_gauge(l.ctx, synth.gauge_field(dims, 0.2, 1 + i))
        bqcd.bq_set_recon(l.ctx, "single", 12)
        bqcd.bq_set_fp64_arith(l.ctx, fp64_arith)
        lats.append(l)
        bs.append(torch.from_numpy(synth.gaussian_spinor(l.Vh, 900 + i)).cuda())
        xr.append(torch.empty_like(bs[-1]))
    ctxs = [l.ctx for l in lats]
    bqcd.bq_solve_cg_batch(ctxs, xr, bs, **kw)
    st_r, ms_r = _timed(torch, lambda: bqcd.bq_solve_cg_batch(ctxs, xr, bs, **kw))
    st_q, ms_q = _timed(torch, lambda: [bqcd.bq_solve_cg(c, x, bb, **kw) for c, x, bb in zip(ctxs, xr, bs)])
    out["ragged_4_lattices"] = {"batched_ms": ms_r, "sequential_ms": ms_q, "speedup": ms_q / ms_r,
                                "max_true_residual": max(s_["true_residual"] for s_ in st_r)}
    for l in lats:
        l.close()
    return out


def batched_apply_roofline(torch, bqcd, lat, nrhs=12, reps=10):
    """The batched hopping-term kernels alone: Mhat^dag Mhat of nrhs Gaussian
    sources in one bq_apply_mdagm_batch call (FP32, 12-real links), CUDA events
    around every launch, for each right-hand-side mapping. Algorithmic bytes per
    launch: links and clover once per site of a unit, spinors per right-hand side."""
    from paper_1711_03836_gb300 import synth

    peak, _ = measured_peaks()
    ins = [lat.pack(synth.gaussian_spinor(lat.Vh, 1200 + i), "single") for i in range(nrhs)]
    outs = [lat.spinor("single") for _ in range(nrhs)]
    res = {"peak_GB/s": peak}
    names = {-3: "tile_4_blocks", -4: "tile_5_blocks", -5: "tile_6_blocks", -1: "block_interleaved",
             -2: "warp_per_rhs", 4: "warp_interleaved_4"}
    for mapping in (-3, -4, -5, -1, -2, 4):
        bqcd.bq_set_batch_mapping(lat.ctx, mapping)
        for _ in range(3):
            bqcd.bq_apply_mdagm_batch([lat.ctx] * nrhs, outs, ins, "single")
        bqcd.bq_reset_counters(lat.ctx, timing=True)
        for _ in range(reps):
            bqcd.bq_apply_mdagm_batch([lat.ctx] * nrhs, outs, ins, "single")
        c = bqcd.bq_get_counters(lat.ctx)
        r = {}
        for epi, en in ((1, "dhop_clovinv"), (2, "dhop_xpay")):
            n = c["dslash_launches"][1][epi]
            ms = c["dslash_ms"][1][epi] / max(n, 1)
            gbs = c["dslash_bytes"][1][epi] / max(n, 1) / (ms * 1e-3) / 1e9
            r[en] = {"us_per_launch": ms * 1e3, "GB/s": gbs, "frac": gbs / peak,
                     "bytes_per_launch": c["dslash_bytes"][1][epi] / max(n, 1)}
        r["mdagm_us"] = 2 * (r["dhop_clovinv"]["us_per_launch"] + r["dhop_xpay"]["us_per_launch"])
        res[names[mapping]] = r
    bqcd.bq_set_batch_mapping(lat.ctx, 0)
    return res


def full_system_extras(torch, bqcd, fp64_arith):
    """M x = b on the whole 24^3x48 lattice with chemical potential mu = 0.1
    (Mhat not gamma_5-hermitian): BiCGstab on Mhat against CG on Mhat^dag Mhat,
    both mixed (FP32 inner, FP64 outer) and BiCGstab in plain FP64, to a true
    full-lattice FP64 residual 1e-10. kappa = 0.12: the synthetic fields are
    close to free, whose critical kappa is 1/8; at the configurations' 0.135 the
    spectrum of Mhat surrounds the origin and BiCGstab diverges."""
    from paper_1711_03836_gb300 import synth

    wl = WORKLOADS["24^3x48"]
    lat = bqcd.Lattice(wl["dims"], 0.12, wl["csw"], 0.1, -1.0)
    bqcd.bq_set_gauge(lat.ctx, synth.gauge_field(wl["dims"], wl["eps"], wl["seed"]))
    bqcd.bq_set_recon(lat.ctx, "single", 12)
    bqcd.bq_set_fp64_arith(lat.ctx, fp64_arith)
    b_e = torch.from_numpy(synth.gaussian_spinor(lat.Vh, 601)).cuda()
    b_o = torch.from_numpy(synth.gaussian_spinor(lat.Vh, 602)).cuda()
    x_e, x_o = torch.empty_like(b_e), torch.empty_like(b_o)
    out = {}
    for name, method, prec in (("bicgstab_mixed", "bicgstab", "single"), ("cg_normal_mixed", "cg", "single"),
                               ("bicgstab_fp64", "bicgstab", "double")):
        kw = dict(method=method, tol=1e-10, precision=prec, delta=1e-3 if method == "cg" else 1e-2)
        bqcd.bq_solve_full(lat.ctx, x_e, x_o, b_e, b_o, **kw)
        st, ms = _timed(torch, lambda: bqcd.bq_solve_full(lat.ctx, x_e, x_o, b_e, b_o, **kw))
        out[name] = {"ms": ms, "iterations": st["iterations"], "dslash_calls": st["dslash_calls"],
                     "true_residual": st["true_residual"]}
    # stochastic traces: 8 Z2 noise vectors (16 full-lattice solves) in one batched call
    # against the same 16 solves one full-system solve at a time
    etas = [(torch.from_numpy(synth.z2_noise(lat.Vh, 610 + 2 * n)).cuda(),
             torch.from_numpy(synth.z2_noise(lat.Vh, 611 + 2 * n)).cuda()) for n in range(8)]
    tkw = dict(tol=1e-10, precision="single", delta=1e-3)
    bqcd.bq_trace_samples(lat.ctx, [e for e, _ in etas], [o for _, o in etas], **tkw)
    (smp, tst), ms_t = _timed(torch, lambda: bqcd.bq_trace_samples(lat.ctx, [e for e, _ in etas],
                                                                   [o for _, o in etas], **tkw))

    def one_by_one():
        for e, o in etas:
            for dag in (False, True):
                bqcd.bq_solve_full(lat.ctx, x_e, x_o, e, o, method="cg", dagger=dag, **tkw)
    _, ms_seq = _timed(torch, one_by_one)
    out_t = {"batched_ms": ms_t, "one_solve_at_a_time_ms": ms_seq, "speedup": ms_seq / ms_t,
             "worst_true_residual": max(s_["true_residual"] for s_ in tst),
             "Tr_Minv_estimate": [float(smp[:, 0].real.mean()), float(smp[:, 0].imag.mean())],
             "Tr_g5Minv_estimate": [float(smp[:, 1].real.mean()), float(smp[:, 1].imag.mean())],
             "Tr_MdagM_inv_estimate": float(smp[:, 2].real.mean())}
    lat.close()
    return {"full_system_24^3x48_kappa0.12_mu0.1": out, "traces_8_noise_24^3x48_kappa0.12_mu0.1": out_t}


def aggregate_ranks(ms, nbytes, device):
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([float(nbytes)], device=device, dtype=torch.float64)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())


def summarize(st):
    sts = st if isinstance(st, list) else [st]
    return {"systems": len(sts), "iterations": max(x["iterations"] for x in sts),
            "reliable_updates": max(x["reliable_updates"] for x in sts),
            "true_residual": max(x["true_residual"] for x in sts),
            "converged": int(all(x["converged"] for x in sts))}


def make_step(args, torch, bqcd, synth, lat, b_dev, x_dev, solve_kw, field_inputs):
    """The timed step of each mode; returns (callable, extra lattices to close)."""
    ctx = lat.ctx
    if args.mode == "qed2x4":
        wl = WORKLOADS[args.workload]
        U, A = field_inputs
        other = bqcd.Lattice(wl["dims"], wl["kappa"], wl["csw"], wl["mu"], -1.0, wl["charges"][1])
        bqcd.bq_set_gauge(other.ctx, U)
        bqcd.bq_set_u1(other.ctx, A)
        bqcd.bq_set_fp64_arith(other.ctx, args.fp64_arith)
        bs = [torch.from_numpy(synth.gaussian_spinor(lat.Vh, 700 + i)).cuda() for i in range(8)]
        xs = [torch.empty_like(b) for b in bs]
        ctxs = [ctx] * 4 + [other.ctx] * 4
        return (lambda: bqcd.bq_solve_cg_batch(ctxs, xs, bs, **solve_kw)), [other]
    if args.mode == "cg":
        return (lambda: bqcd.bq_solve_cg(ctx, x_dev, b_dev, **solve_kw)), []
    if args.mode == "batch12":
        srcs = [torch.from_numpy(synth.point_source(lat.Vh, 0, s, c)).cuda() for s in range(4) for c in range(3)]
        xs = [torch.empty_like(b) for b in srcs]
        return (lambda: bqcd.bq_solve_cg_batch([ctx] * 12, xs, srcs, **solve_kw)), []
    if args.mode == "multishift10":
        shifts = [10.0 ** (-4 + 4 * k / 9) for k in range(10)]
        xk = [torch.empty_like(b_dev) for _ in shifts]
        kw = {k: v for k, v in solve_kw.items() if k != "max_iter"}
        return (lambda: bqcd.bq_solve_multishift_cg(ctx, xk, b_dev, shifts, **kw)), []
    if args.mode == "blockms4x10":
        shifts = [10.0 ** (-4 + 4 * k / 9) for k in range(10)]
        b4 = [torch.from_numpy(synth.gaussian_spinor(lat.Vh, 780 + r)).cuda() for r in range(4)]
        x4 = [[torch.empty_like(b_dev) for _ in shifts] for _ in b4]
        kw = {k: v for k, v in solve_kw.items() if k != "max_iter"}
        return (lambda: bqcd.bq_solve_multishift_cg_block(ctx, x4, b4, shifts, **kw)), []
    if args.mode == "full_cg":
        b_o = torch.from_numpy(synth.gaussian_spinor(lat.Vh, 602)).cuda()
        x_o = torch.empty_like(b_o)
        return (lambda: bqcd.bq_solve_full(ctx, x_dev, x_o, b_dev, b_o, method="cg", **solve_kw)), []
    if args.mode == "traces8":
        etas = [(torch.from_numpy(synth.z2_noise(lat.Vh, 610 + 2 * n)).cuda(),
                 torch.from_numpy(synth.z2_noise(lat.Vh, 611 + 2 * n)).cuda()) for n in range(8)]
        return (lambda: bqcd.bq_trace_samples(ctx, [e for e, _ in etas], [o for _, o in etas], **solve_kw)[1]), []
    # ragged: the workload lattice plus 8^4, 12^4 and 16^3x32, in one batched solve
    lats, bs, xr = [lat], [b_dev], [x_dev]
    for i, dims in enumerate([(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32)]):
        l = bqcd.Lattice(dims, 0.1350, 1.7, 0.0, -1.0)
        bqcd.bq_set_gauge(l.ctx, synth.gauge_field(dims, 0.2, 1 + i))
        bqcd.bq_set_recon(l.ctx, "single", 12)
        bqcd.bq_set_recon(l.ctx, "half", 12)
        bqcd.bq_set_fp64_arith(l.ctx, args.fp64_arith)
        lats.append(l)
        bs.append(torch.from_numpy(synth.gaussian_spinor(l.Vh, 900 + i)).cuda())
        xr.append(torch.empty_like(bs[-1]))
    ctxs = [l.ctx for l in lats]
    return (lambda: bqcd.bq_solve_cg_batch(ctxs, xr, bs, **solve_kw)), lats[1:]


def extras(args, ctx, lat, b, b_dev, x_dev, solve_kw, mixed_ms, torch, bqcd):
    out = {}
    Vh = lat.Vh
    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region)
    b_host = torch.from_numpy(b).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    bqcd.bq_reset_counters(ctx, timing=False)
    n_e2e = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        bqcd.bq_solve_cg(ctx, x_host, b_host, **solve_kw)
    t1 = time.perf_counter()
    cnt = bqcd.bq_get_counters(ctx)
    e2e_bytes = sum(sum(r) for r in cnt["dslash_bytes"])
    out["e2e"] = {"value": e2e_bytes / (t1 - t0) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": Vh * 192,
                  "d2h_bytes_per_step": Vh * 192, "ms_per_step": (t1 - t0) / n_e2e * 1e3}

    # ---- plain FP64 CG on the same system, with the FP64 units and with double-float arithmetic
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fp64 = {}
    for mode in ("native", "df64"):
        bqcd.bq_set_fp64_arith(ctx, mode)
        bqcd.bq_solve_cg(ctx, x_dev, b_dev, tol=1e-10, precision="double", check_every=8, max_iter=20000)
        e0.record()
        st64 = bqcd.bq_solve_cg(ctx, x_dev, b_dev, tol=1e-10, precision="double", check_every=8, max_iter=20000)
        e1.record()
        torch.cuda.synchronize()
        fp64[mode] = (e0.elapsed_time(e1), st64)
    bqcd.bq_set_fp64_arith(ctx, args.fp64_arith)
    # the same solve with FP16 storage in the inner iteration (12-real links, per-site FP32 scale)
    half_kw = dict(tol=1e-10, precision="half", delta=1e-3, check_every=args.check_every, max_iter=20000)
    bqcd.bq_solve_cg(ctx, x_dev, b_dev, **half_kw)
    e0.record()
    st_h = bqcd.bq_solve_cg(ctx, x_dev, b_dev, **half_kw)
    e1.record()
    torch.cuda.synchronize()
    out["cg_fp16_inner"] = {"ms": e0.elapsed_time(e1), "delta": 1e-3, "iterations": st_h["iterations"],
                            "reliable_updates": st_h["reliable_updates"], "true_residual": st_h["true_residual"]}
    out["cg"] = {"fp64_native_ms": fp64["native"][0], "fp64_df64_ms": fp64["df64"][0], "mixed_ms": mixed_ms,
                 "speedup_mixed_vs_fp64_native": fp64["native"][0] / mixed_ms,
                 "speedup_mixed_vs_fp64_df64": fp64["df64"][0] / mixed_ms,
                 "fp64_iterations": fp64["native"][1]["iterations"],
                 "fp64_true_residual": fp64["native"][1]["true_residual"],
                 "fp64_df64_true_residual": fp64["df64"][1]["true_residual"]}

    # ---- hopping-term bandwidth sweep (plain D_hop, inputs larger than L2)
    sweep = {}
    for prec, recon, arith in (("double", 18, "native"), ("double", 12, "native"), ("double", 18, "df64"),
                               ("single", 18, None), ("single", 12, None), ("single", 8, None),
                               ("half", 18, None), ("half", 12, None), ("half", 8, None)):
        bqcd.bq_set_recon(ctx, prec, recon)
        if arith:
            bqcd.bq_set_fp64_arith(ctx, arith)
        src = lat.pack(b, prec)
        dst = lat.spinor(prec)
        for _ in range(3):
            bqcd.bq_apply_dhop(ctx, dst, src, 1, 0, prec)
        n = 20
        e0.record()
        for i in range(n):
            bqcd.bq_apply_dhop(ctx, dst, src, i & 1, 0, prec)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / n * 1e-3
        pid = PREC_ID[prec]
        byts = (8 * link_b(pid, recon) + 2 * SPINOR_B[pid]) * Vh
        sweep[f"{prec}_r{recon}" + (f"_{arith}" if arith else "")] = {
            "GB/s": byts / t / 1e9, "GFLOP/s": 1320.0 * Vh / t / 1e9, "us": t * 1e6}
    bqcd.bq_set_recon(ctx, "double", 18)
    bqcd.bq_set_fp64_arith(ctx, args.fp64_arith)
    bqcd.bq_set_recon(ctx, "single", 12)
    bqcd.bq_set_recon(ctx, "half", 12)
    out["dslash_sweep"] = sweep

    fp64_peak, fp64_src = measured_fp64_peak()
    hbm_peak, _ = measured_peaks()
    out["fp64_peak"] = {"GFLOP/s": fp64_peak, "source": fp64_src}
    for k, v in sweep.items():
        if k.startswith("double"):
            # 1320 flops per 1536 (r18) / 1152 (r12) bytes: at the HBM peak that would need
            # 5.8 / 7.8 TFLOP/s, so min(HBM, FP64) binds at the FP64 rate for the FP64 units
            bound = min(hbm_peak, fp64_peak * v["GB/s"] / max(v["GFLOP/s"], 1e-9))
            v["frac_of_min_hbm_fp64"] = v["GB/s"] / bound
            v["frac_of_fp64_peak"] = v["GFLOP/s"] / fp64_peak

    # ---- gauge-side setup: one stout step of every link, clover log det of each parity
    Vfull = 2 * Vh
    U_dev = torch.empty((Vfull, 4, 3, 3), dtype=torch.complex128, device="cuda")
    bqcd.bq_set_stout(ctx, 0.1, 1)
    bqcd.bq_get_hop_links(ctx, U_dev)  # warm
    bqcd.bq_set_stout(ctx, 0.0, 0)
    bqcd.bq_set_stout(ctx, 0.1, 1)
    _, ms_stout = _timed(torch, lambda: bqcd.bq_get_hop_links(ctx, U_dev))
    bqcd.bq_set_stout(ctx, 0.0, 0)
    _, ms_copy = _timed(torch, lambda: bqcd.bq_get_hop_links(ctx, U_dev))
    del U_dev
    _, ms_clov = _timed(torch, lambda: bqcd.bq_build_clover(ctx))
    bqcd.bq_clover_logdet(ctx, 1)
    (ld, neg), ms_ld = _timed(torch, lambda: bqcd.bq_clover_logdet(ctx, 1))
    out["gauge_setup"] = {"stout_step_ms": ms_stout - ms_copy, "stout_plus_link_copy_ms": ms_stout,
                          "stout_GB/s_links_in_out": 2 * Vfull * 4 * 144 / ((ms_stout - ms_copy) * 1e-3) / 1e9,
                          "clover_build_and_invert_ms": ms_clov, "clover_logdet_odd_ms": ms_ld, "clover_logdet_odd": ld, "negative_blocks": neg}

    # ---- batching (row a9) and multishift (row a8), each against the same work done one system at a time
    out["batched"] = batched_extras(torch, bqcd, args.fp64_arith)
    out.update(full_system_extras(torch, bqcd, args.fp64_arith))

    # ---- the configuration-2 lattice (16^3x32, mu = 0 and 0.1): fields fit in L2
    out["config2_16^3x32"] = config2_extras(torch, bqcd, args.fp64_arith)

    # ---- CPU oracle on the host cores: median of 5 Mhat^dag Mhat applies on the workload
    # lattice, and the oracle's D_hop and CG on configurations 1 and 2
    import oracle

    wl = WORKLOADS[args.workload]
    op, bb, Vh_o = oracle_setup(wl)
    gbs, t_step = oracle_gbs(op, bb, Vh_o, 5, 1, median=True)
    out["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
                           "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                           "sample": f"median of 5 FP64 Mhat^dag Mhat applies on the full {args.workload} "
                                     f"lattice, {t_step:.2f} s each"}
    out["cpu_oracle_configs"] = oracle_config_timings(out["config2_16^3x32"])
    return out


def oracle_config_timings(gpu_cfg2):
    """The oracle's D_hop (median of 5) and CG solves on configurations 1 (8^4) and 2
    (16^3x32, mu = 0 and 0.1) on the host cores: CG timed in full on 8^4 (median
    of 5); on 16^3x32 one Mhat^dag Mhat apply (median of 5) times the GPU solve's
    iteration count, labelled extrapolated."""
    import oracle
    from paper_1711_03836_gb300 import synth

    res = {"cores": oracle.num_threads(), "nproc": os.cpu_count(), "cpu_model": cpu_model()}
    for name, wl_name, mu in (("8^4", "8^4", 0.0), ("16^3x32_mu0", "16^3x32", 0.0), ("16^3x32_mu0.1", "16^3x32", 0.1)):
        wl = dict(WORKLOADS[wl_name], mu=mu)
        op, b, Vh = oracle_setup(wl)
        U = op.U
        psi = synth.gaussian_spinor(Vh, 5)
        ts = []
        for _ in range(6):
            t0 = time.perf_counter()
            oracle.dhop(op.p, U, None, psi, 0)
            ts.append(time.perf_counter() - t0)
        t_d = statistics.median(ts[1:])
        r = {"dhop_ms": t_d * 1e3, "dhop_GB/s": 1536.0 * Vh / t_d / 1e9, "dhop_GFLOP/s": 1320.0 * Vh / t_d / 1e9}
        if wl_name == "8^4":
            ts = []
            its = 0
            for _ in range(6):
                t0 = time.perf_counter()
                _, its = op.cg(b, tol=1e-10)
                ts.append(time.perf_counter() - t0)
            r.update({"cg_ms": statistics.median(ts[1:]) * 1e3, "cg_iterations": int(its)})
        else:
            _, t_m = oracle_gbs(op, b, Vh, 5, 1, median=True)
            key = "mu0" if mu == 0.0 else "mu0.1"
            its = gpu_cfg2.get(key, {}).get("fp64_iterations")
            if its:
                r.update({"cg_ms_extrapolated": t_m * its * 1e3, "cg_iterations_of_gpu_fp64_solve": its,
                          "mdagm_apply_ms": t_m * 1e3, "note": "extrapolated: one apply x iteration count"})
        res[name] = r
    return res


def config2_extras(torch, bqcd, fp64_arith):
    """16^3x32, kappa 0.1350, c_SW 1.7, links exp(i 0.2 A): FP64 vs FP32 D_hop
    (plain, FP64 units, double-float, FP32 r18 / r12) and the mixed CG (FP32
    inner, FP64 reliable update at every 1e-3 drop) against plain FP64 CG, at
    mu = 0 and mu = 0.1. The FP64 links (75 MB), clover and spinors fit in the
    129 MB L2 with room to spare, so these figures are L2-resident: GB/s above
    the HBM peak are possible here and are not HBM figures."""
    from paper_1711_03836_gb300 import synth

    wl = WORKLOADS["16^3x32"]
    res = {"l2": "L2-resident (FP64 links 75 MB, FP32 links 25 MB, one FP32 spinor 6 MB)"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    U = synth.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    for mu in (0.0, 0.1):
        lat = bqcd.Lattice(wl["dims"], wl["kappa"], wl["csw"], mu, -1.0)
        ctx = lat.ctx
        bqcd.bq_set_gauge(ctx, U)
        bqcd.bq_set_fp64_arith(ctx, fp64_arith)
        b = synth.gaussian_spinor(lat.Vh, wl["seed"] + 1000)
        b_dev = torch.from_numpy(b).cuda()
        x_dev = torch.empty_like(b_dev)
        r = {}
        sweep = {}
        for prec, recon, arith in (("double", 18, "native"), ("double", 18, "df64"), ("single", 18, None),
                                   ("single", 12, None)):
            bqcd.bq_set_recon(ctx, prec, recon)
            if arith:
                bqcd.bq_set_fp64_arith(ctx, arith)
            src, dst = lat.pack(b, prec), lat.spinor(prec)
            for _ in range(3):
                bqcd.bq_apply_dhop(ctx, dst, src, 1, 0, prec)
            n = 50
            e0.record()
            for i in range(n):
                bqcd.bq_apply_dhop(ctx, dst, src, i & 1, 0, prec)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / n * 1e-3
            pid = PREC_ID[prec]
            sweep[f"{prec}_r{recon}" + (f"_{arith}" if arith else "")] = {
                "GB/s": (8 * link_b(pid, recon) + 2 * SPINOR_B[pid]) * lat.Vh / t / 1e9,
                "GFLOP/s": 1320.0 * lat.Vh / t / 1e9, "us": t * 1e6}
        bqcd.bq_set_fp64_arith(ctx, fp64_arith)
        bqcd.bq_set_recon(ctx, "single", 12)
        r["dslash_sweep"] = sweep
        kw = dict(tol=1e-10, check_every=8, max_iter=20000)
        for name, prec in (("mixed", "single"), ("fp64", "double")):
            bqcd.bq_solve_cg(ctx, x_dev, b_dev, precision=prec, delta=1e-3, **kw)
            e0.record()
            st = bqcd.bq_solve_cg(ctx, x_dev, b_dev, precision=prec, delta=1e-3, **kw)
            e1.record()
            torch.cuda.synchronize()
            r[f"{name}_ms"] = e0.elapsed_time(e1)
            r[f"{name}_iterations"] = st["iterations"]
            r[f"{name}_true_residual"] = st["true_residual"]
        r["speedup_mixed_vs_fp64"] = r["fp64_ms"] / r["mixed_ms"]
        res["mu0" if mu == 0.0 else "mu0.1"] = r
        lat.close()
    return res


if __name__ == "__main__":
    sys.exit(main())
