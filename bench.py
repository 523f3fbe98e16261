#!/usr/bin/env python3
"""Throughput of the skeletonized-FMM apply (Algorithm 2) on GB300.

Metric: Mpts*RHS/s = N * nrhs / T_apply for 3D Laplace, N = 2^20 points
uniform in [0,1]^3, q ~ N(0,1), leaf 128, ID tolerance 1e-6 (the plan is
built once, outside the timed region). One step = one apply of all 32
right-hand sides in the batched FP32 tensor-core path (``--precision``), the
operators and charges resident in HBM. Next to it, on the same plan: the
plain FP64 single-RHS apply (the comparator), relative errors of both against
the oracle's FP64 direct sum on 4096 sampled targets, an end-to-end figure
through the C-ABI with pinned host buffers, the dominant kernel against its
roofline, and the oracle timed on the host cores.

Multi-GPU: the apply does not shard across GPUs here; every rank runs an
independent replica (its own point set) and ``value`` sums the replicas.

``--impl reference`` times the oracle (the FP64 direct sum in plain C) on a
bounded sample of targets per step, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpts·RHS/s, 3D Laplace apply N=1M, err≤1e-6: batched FP32 TC vs plain FP64"
UNIT = "Mpts·RHS/s"
SM_COUNT = 152
MUFU_PER_SM_CLK = 16      # MUFU (rsqrt) results per SM per clock
FP32_PER_SM_CLK = 128     # FP32 lane operations per SM per clock (a paired instruction counts as two)
# FP32 operations per complex kernel evaluation in tc_cnear_kernel, counted
# from its source (tc_ceval16 + tc_sincos2): differences 3, r^2 3, r with one
# Newton step 5, kappa r 1, reduction 3 + 2, z 1, sin 5, cos 5, G_r / G_i 2,
# TF32 split 8 (touching-leaf tiles add 9, not counted)
FP32_OPS_HELMHOLTZ_TC = 38


# --workload name -> workload in paper_2310_16668_gb300.workloads
WORKLOAD_KEYS = {"laplace3d": "LAPLACE3D_1M", "sphere_cluster": "LAPLACE3D_ADAPTIVE_4M",
                 "helmholtz3d": "HELMHOLTZ3D_1M", "laplace2d": "LAPLACE2D_16K", "curves2d": "CURVES2D_256",
                 "helmholtz2d": "HELMHOLTZ2D_1M"}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="laplace3d", choices=list(WORKLOAD_KEYS),
                   help="laplace3d: the headline (3D Laplace, N = 2^20 uniform); sphere_cluster: 3D Laplace, "
                        "N = 2^22 on a sphere plus a Gaussian cluster; helmholtz3d: kappa = 25, N = 2^20; "
                        "laplace2d: N = 16384; curves2d: 256 independent 2D point sets on closed curves, "
                        "applied as one CUDA graph; helmholtz2d: kappa = 100, N = 2^20 uniform in 2D")
    p.add_argument("--precision", default=None, choices=["fp32_tc", "fp32", "fp64"],
                   help="default: fp32_tc, fp32 (complex64) for 2D Helmholtz")
    p.add_argument("--nrhs", type=int, default=None, help="default 32 (curves2d: 4)")
    p.add_argument("--tol", type=float, default=None)
    p.add_argument("--n", type=int, default=None, help="override N (testing only)")
    p.add_argument("--build", default="host", choices=["host", "device"],
                   help="where Algorithm 1 runs (outside the timed region either way)")
    p.add_argument("--store-tiles", type=int, default=0, choices=[0, 1, 2],
                   help="stored-operator mode at build: 1 every tile's kernel values, 2 the symmetric store "
                        "(shared blocks once); read by every apply")
    p.add_argument("--tune", default="auto", choices=["auto", "none"],
                   help="auto: skel_autotune after the build (per-level up/down variants; stored or on-the-fly "
                        "kernel tiles, chosen by measurement); none: the default rules, tiles on the fly")
    p.add_argument("--updown-tc", action="store_true",
                   help="upward / downward skeleton GEMMs on the tensor cores (skel_options.updown_tc)")
    p.add_argument("--updown-shape", type=int, default=None,
                   help="force the FP32 up/down launch shape on every level (skel_test_set_updown code: 1, 2, 4, 8 "
                        "plain kernel warps; 17, 18, 20, 24 the CTA-wide kernel); same result, for profiling")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha(kernel: str = "") -> str:
    """Hash of the files that define a device kernel's code (the kernels and
    the structures they read; the complex tensor-core kernel adds its own
    header); a committed traffic figure counts only while it matches."""
    h = hashlib.sha256()
    files = ("skel_kernels.cuh", "tc_kernels.cuh", "host.h")
    if kernel == "tc_cnear_kernel":
        files += ("tc_complex.cuh",)
    for f in files:
        p = os.path.join(ROOT, "paper_2310_16668_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, precision: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from a committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    sha = kernel_source_sha(kernel)
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    pat = re.compile(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+kernel:\s*(\S+)\s+precision:\s*(\S+)\s+"
                     r"source_sha:\s*([0-9a-f]+)\s+workload:\s*(\S+)")
    for f in sorted(os.listdir(d)):
        if not f.endswith((".md", ".txt")):
            continue
        for m in pat.finditer(open(os.path.join(d, f)).read()):
            if (m.group(2), m.group(3), m.group(4), m.group(5)) == (kernel, precision, sha, workload):
                return float(m.group(1))
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except ValueError:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s independent replica (its own point set)."""
    return base + 17 * rank


def max_over_ranks(value: float, dist, device) -> float:
    """The largest `value` over all ranks (the job is as slow as its slowest rank)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n: int, nrhs: int, world: int, ms_step: float) -> float:
    """Mpts*RHS/s of the whole job: every rank applies its own n x nrhs problem per step."""
    return n * nrhs * world / (ms_step * 1e-3) / 1e6


def oracle_direct_sample(kind, x, q0, targets, kappa=0.0):
    """The oracle's FP64 (complex128) direct sum at `targets` (cpu_baseline leg)."""
    from oracle import direct
    t0 = time.perf_counter()
    u = direct.direct_sum(kind, x, q0, targets=targets, kappa=kappa)
    return u, time.perf_counter() - t0, direct.num_threads()


def roofline(info, phases, clk, prec, pairs, kind="laplace3d", workload=""):
    """The dominant kernel against its roofline: the main translation kernel,
    timed by the plan's own CUDA events on the launching stream inside the
    timed region (skel_set_profiling); the CUDA-core launch for the small
    non-leaf boxes is outside that span. On the fly it is bound by the MUFU
    unit (one operation per kernel evaluation); reading stored tiles, by
    HBM."""
    if prec == "fp32_tc" and kind == "helmholtz3d":
        kname, units = "tc_cnear_kernel", info["pairs_tc"]
        unit_note = "skel_info pairs_tc: kept complex kernel evaluations of the tensor-core items"
    elif prec == "fp32_tc":
        kname, units = "tc_near_kernel", info["pairs_tc"]
        unit_note = "skel_info pairs_tc: kept kernel evaluations of the tensor-core items"
    else:
        kname, units = "near_kernel", pairs
        unit_note = "skel_info pairs_direct + pairs_far"
    n_near = phases["main_launches"] / phases["n_applies"]
    near_ms_per_launch = phases["main_near"] / phases["main_launches"]
    achieved = units / (near_ms_per_launch * 1e-3) / 1e9
    sm_mhz = clk.get("sm_mhz") or 2070.0
    # one MUFU operation per evaluation (reciprocal square root in 3D, the
    # logarithm in 2D); for Helmholtz the same figure is an upper bound
    peak = SM_COUNT * MUFU_PER_SM_CLK * sm_mhz * 1e6 / 1e9
    peaks, peaks_kind = measured_peaks()
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
            "frac": achieved / peak, "traffic": ncu_traffic(kname, prec, workload),
            "peak_basis": f"{SM_COUNT} SMs x {MUFU_PER_SM_CLK} MUFU ops/clk x median SM clock under load "
                          f"({sm_mhz:.0f} MHz), one MUFU op per kernel evaluation",
            "per_launch_ms": near_ms_per_launch, "launches_per_step": n_near,
            "algorithmic_units": f"{units} kernel evaluations per launch ({unit_note})"}
    if kname == "tc_cnear_kernel":
        # complex: one MUFU operation but ~38 FP32 operations per evaluation
        # (the sine and cosine are polynomials): the FP32 pipe is the bound
        peak = SM_COUNT * FP32_PER_SM_CLK * sm_mhz * 1e6 / FP32_OPS_HELMHOLTZ_TC / 1e9
        roof.update({"peak": peak, "frac": achieved / peak,
                     "peak_basis": f"{SM_COUNT} SMs x {FP32_PER_SM_CLK} FP32 ops/clk x median SM clock under load "
                                   f"({sm_mhz:.0f} MHz) / {FP32_OPS_HELMHOLTZ_TC} FP32 ops per complex evaluation"})
    stored = prec == "fp32_tc" and info["stored_tile_bytes"] > 0
    if stored and info["store_mode"] == 1:
        # per-tile store, HBM-bound: the algorithmic bytes are 4 B per kept
        # kernel evaluation (pairs_tc, each value read once per 32-column
        # pass) plus the rows of U the launch writes; the stored bytes beyond
        # that (zero padding of ragged tiles, masked entries) and the chunks'
        # B blocks (8 KB per tile, mostly L2 hits) are overhead, reported
        # beside the figure
        kname = "tc_stored_kernel"
        alg_bytes = 4 * info["pairs_tc"] + info["n_index"] * 32 * 4
        traffic = ncu_traffic(kname, prec, workload)
        roof.update({"kernel": kname, "bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                     "achieved": alg_bytes / (near_ms_per_launch * 1e-3) / 1e9,
                     "traffic": traffic,
                     "peak_basis": f"{peaks_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_units": f"{alg_bytes} bytes per launch (4 B x pairs_tc {info['pairs_tc']} "
                                          f"+ U rows {info['n_index']} x 32 x 4)",
                     "stored_tile_bytes": info["stored_tile_bytes"],
                     "stored_over_algorithmic": info["stored_tile_bytes"] / (4 * info["pairs_tc"]),
                     "traffic_over_algorithmic": (traffic / alg_bytes) if traffic else None,
                     "evaluation_rate_gpair_s": achieved})
        roof["frac"] = roof["achieved"] / roof["peak"]
    elif stored:
        # stored-operator mode, HBM-bound: the algorithmic bytes are 4 B per
        # kept kernel evaluation (pairs_tc, each value read once per 32-column
        # pass) plus the rows of U the launch writes; the stored bytes beyond
        # that (zero padding of ragged tiles, masked entries) and the chunks'
        # B blocks (8 KB per tile, mostly L2 hits) are overhead, reported
        # beside the figure, not counted as useful work
        # symmetric store: a kernel value shared by two tiles (G(e, f) =
        # G(f, e)) is held and read once, so the minimum is 4 B per distinct
        # kept value (skel_info pairs_stored), not per evaluation
        kname = "tc_sym_kernel"
        alg_bytes = 4 * info["pairs_stored"] + info["n_index"] * 32 * 4
        traffic = ncu_traffic(kname, prec, workload)
        roof.update({"kernel": kname, "bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                     "achieved": alg_bytes / (near_ms_per_launch * 1e-3) / 1e9,
                     "traffic": traffic,
                     "peak_basis": f"{peaks_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_units": f"{alg_bytes} bytes per launch (4 B x pairs_stored {info['pairs_stored']} "
                                          f"distinct kept kernel values of pairs_tc {info['pairs_tc']} evaluations "
                                          f"+ U rows {info['n_index']} x 32 x 4)",
                     "stored_tile_bytes": info["stored_tile_bytes"],
                     "stored_over_algorithmic": info["stored_tile_bytes"] / (4 * info["pairs_stored"]),
                     "traffic_over_algorithmic": (traffic / alg_bytes) if traffic else None,
                     "evaluation_rate_gpair_s": achieved})
        roof["frac"] = roof["achieved"] / roof["peak"]
    if prec == "fp32_tc":
        # the same launch against the tensor pipe: algorithmic 2 flops per
        # evaluation and right-hand side (32 per launch); the pipe issues 3
        # TF32 products (hi.hi + hi.lo + lo.hi) over full 128 x 32 tiles
        # (complex: 8 real flops per evaluation and complex right-hand side,
        # 16 per launch, the same 2 x 32 real flops; 6 products issued)
        tc_tflops = units * 2 * 32 / (near_ms_per_launch * 1e-3) / 1e12
        n_prod = 6 if kname == "tc_cnear_kernel" else 3
        issued = info["n_tc_tiles"] * 128 * 32 * 32 * 2 * n_prod / (near_ms_per_launch * 1e-3) / 1e12
        tf32_peak = peaks["bf16_tflops"] * 0.5
        roof["tensor"] = {"achieved": tc_tflops, "peak": tf32_peak, "unit": "TFLOP/s", "frac": tc_tflops / tf32_peak,
                          "issued_tflops": issued,
                          "peak_basis": f"TF32 = 0.5 x {peaks_kind} bf16 burst ({peaks['bf16_tflops']} TFLOP/s)"}
    return roof


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import dataclasses
    from oracle import direct
    from paper_2310_16668_gb300 import workloads as W
    if args.workload == "curves2d":
        # the oracle on the largest of the curve sets
        cs = W.CURVES2D_256
        i = int(np.argmax(cs.sizes()))
        wl0 = W.Workload(cs.name, "laplace2d", 2, int(cs.sizes()[i]), cs.leaf, cs.tol, 1, charges="uniform")
        x = W.points_curve(wl0.n, cs.seed * 100003 + i)
        q0 = np.ascontiguousarray(cs.make_charges(i, wl0.n, 1)[:, 0])
        wl, n = wl0, wl0.n
    else:
        wl0 = getattr(W, WORKLOAD_KEYS[args.workload])
        n = args.n or wl0.n
        wl = dataclasses.replace(wl0, n=n)
        x = wl.make_points()
        q0 = np.ascontiguousarray(wl.make_charges(1)[:, 0])
    per_step = max(16, min(1024, int(1e9 // n)))       # ~1e9 pair evaluations per step
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        direct.direct_sum(wl.kernel, x, q0, targets=rng.choice(n, per_step, replace=False), kappa=wl.kappa)
    times = []
    for _ in range(args.steps):
        tg = rng.choice(n, per_step, replace=False)
        t0 = time.perf_counter()
        direct.direct_sum(wl.kernel, x, q0, targets=tg, kappa=wl.kappa)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    value = per_step * args.steps / T / 1e6
    cores = direct.num_threads()
    metric = METRIC if args.workload == "laplace3d" else f"Mpts·RHS/s, {wl0.name} apply"
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl0.name, "N": n, "nrhs": 1, "sample_targets_per_step": per_step,
                   "method": "oracle FP64 direct sum (plain C, OpenMP), throughput extrapolated per target"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random targets x {n} sources x 1 RHS per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_curves(args):
    """Batched 2D Laplace: the 256 independent curve sets merged into one plan
    (skel_merge), so that every phase of the apply is one launch over all
    sets; the forward apply (and forward + adjoint) captured into one CUDA
    graph and replayed. value = total points x right-hand sides / replay
    time. The per-set graph (every set's own apply queued back to back) is
    timed beside it."""
    import torch
    from paper_2310_16668_gb300 import SkelBatch
    from paper_2310_16668_gb300 import workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cs = W.CURVES2D_256
    nrhs = args.nrhs or cs.nrhs
    prec = args.precision or "fp32_tc"
    tol = args.tol or cs.tol
    sets = cs.make_point_sets()
    t0 = time.perf_counter()
    batch = SkelBatch(sets, "laplace2d", tol, cs.leaf, nrhs_max=nrhs)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    fmm = batch.merged(nrhs_max=nrhs)
    t_merge = time.perf_counter() - t0
    tuning = None
    if args.tune == "auto" and prec != "fp64":
        t0 = time.perf_counter()
        try:
            tuning = fmm.autotune(nrhs, allow_store=True)
            tuning["t_tune_s"] = time.perf_counter() - t0
        except Exception as e:                              # keep the untuned plan
            tuning = {"error": str(e)}
    info = fmm.info()
    ntot = int(sum(batch.sizes))
    off = batch.offsets
    rdt = torch.float64 if prec == "fp64" else torch.float32
    qs = [torch.from_numpy(np.ascontiguousarray(cs.make_charges(i, len(x), nrhs).T)).to(dev, rdt)
          for i, x in enumerate(sets)]
    Q = torch.cat(qs, dim=1).contiguous()                   # N x nrhs column-major, sets one after the other
    U = torch.empty_like(Q)
    G = torch.empty_like(Q).normal_()
    V = torch.empty_like(Q)
    stream = torch.cuda.current_stream(dev)

    def capture(adjoint):
        fmm.apply_into(Q, U, nrhs, prec)                    # warm-up outside the capture
        if adjoint:
            fmm.apply_into(G, V, nrhs, prec, transpose=True)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                fmm.apply_into(Q, U, nrhs, prec)
                if adjoint:
                    fmm.apply_into(G, V, nrhs, prec, transpose=True)
        return g

    def timed(g, steps):
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    g_fwd = capture(False)
    g_both = capture(True)
    clocks = ClockSampler(local)
    clocks.start()
    ms_fwd = timed(g_fwd, args.steps)
    clk = clocks.stop()
    ms_both = timed(g_both, args.steps)
    value = ntot * nrhs / (ms_fwd * 1e-3) / 1e6
    # the phases of the same applies, un-captured, timed by the plan's events
    fmm.set_profiling(args.steps)
    for _ in range(args.steps):
        fmm.apply_into(Q, U, nrhs, prec)
    torch.cuda.synchronize()
    phases = fmm.last_timings()
    fmm.set_profiling(0)
    fmm.device_status()
    launches_per_apply = phases["launches"] / phases["n_applies"]
    g_fwd.replay()
    torch.cuda.synchronize()
    # beside it: every set's own apply queued back to back in one graph
    us = [torch.empty_like(q) for q in qs]
    g_sets = batch.capture(qs, us, nrhs, prec)
    ms_sets = timed(g_sets, args.steps)
    torch.cuda.synchronize()
    # the merged plan against the per-set plans: bit for bit unless the
    # merged plan keeps stored blocks (symmetric store: FP32 rounding)
    diff = max(float((us[i] - U[:, off[i]:off[i + 1]]).abs().max() / us[i].abs().max())
               for i in range(len(sets)))
    # end to end through the C-ABI: pinned host buffers, staged by the library
    qh = Q.cpu().pin_memory()
    uh = torch.empty_like(qh).pin_memory()
    fmm.apply_into(qh, uh, nrhs, prec, stream=stream.cuda_stream)
    k = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(k):
        fmm.apply_into(qh, uh, nrhs, prec, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / k
    nbytes = qh.numel() * qh.element_size()
    e2e = {"value": ntot * nrhs / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "ms_per_step": dt * 1e3}
    # errors: the four largest sets, first and last right-hand side, at 1024
    # sampled targets against the oracle's FP64 direct sum
    from oracle import direct
    errs, t_cpu, n_eval = {}, 0.0, 0
    for i in np.argsort(batch.sizes)[-4:]:
        x = sets[i]
        tg = np.sort(np.random.default_rng(int(i)).choice(len(x), min(1024, len(x)), replace=False))
        for r in sorted({0, nrhs - 1}):
            q_r = Q[r, off[i]:off[i + 1]].double().cpu().numpy()
            t1 = time.perf_counter()
            ref = direct.direct_sum("laplace2d", x, q_r, targets=tg)
            t_cpu += time.perf_counter() - t1
            n_eval += len(tg)
            got = U[r, off[i]:off[i + 1]].double().cpu().numpy()[tg]
            errs[f"set{i}_rhs{r}"] = float(np.abs(got - ref).max() / np.abs(ref).max())
    roof = roofline(info, phases, clk, prec, info["pairs_direct"] + info["pairs_far"], "laplace2d", cs.name)
    line = {
        "metric": f"Mpts·RHS/s, {cs.name} batched apply (one merged plan, CUDA graph)", "value": value,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_fwd,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": cs.name, "n_sets": len(sets), "N_total": ntot, "N_min": int(min(batch.sizes)),
                   "N_max": int(max(batch.sizes)), "nrhs": nrhs, "leaf": cs.leaf, "tol": tol,
                   "precision": prec, "t_build_s": t_build, "t_merge_s": t_merge,
                   "l2": f"inputs larger than L2: merged plan {info['device_bytes'] / 1e9:.2f} GB resident",
                   "translations": ({1: "per-tile store", 2: "symmetric store"}.get(info["store_mode"], "kernel on the fly"))},
        "forward_and_adjoint_ms": ms_both,
        "per_set_graph_ms": ms_sets,
        "merged_vs_per_set_maxrel": diff,
        "kernel_launches_per_apply": launches_per_apply,
        "relerr": max(errs.values()),
        "relerr_sets": errs,
        "tuning": tuning,
        "phases_ms_per_step": {k2: v / phases["n_applies"] for k2, v in phases.items()
                               if k2 not in ("launches", "n_applies", "main_launches")},
        "roofline": roof,
        "cpu_baseline": {"value": n_eval / t_cpu / 1e6, "unit": UNIT, "cores": direct.num_threads(),
                         "kind": "oracle", "sample": f"FP64 direct sum at {n_eval} targets of the 4 largest sets"},
        "e2e": e2e,
        "gpu_launches": int(launches_per_apply * args.steps),
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons")},
    }
    print(json.dumps(line), flush=True)
    fmm.close()
    batch.close()
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2310_16668_gb300 import SkelFMM
    from paper_2310_16668_gb300 import workloads as W

    import dataclasses
    wl0 = getattr(W, WORKLOAD_KEYS[args.workload])
    n = args.n or wl0.n
    tol = args.tol or wl0.tol
    nrhs = args.nrhs or 32
    # independent replica per rank: the workload's recipe with its own seed
    wl = dataclasses.replace(wl0, n=n, seed=replica_seed(wl0.seed, rank))
    x = wl.make_points()
    q = wl.make_charges(nrhs)
    cplx = wl.kernel in ("helmholtz3d", "helmholtz2d")
    threads = max(1, (os.cpu_count() or 1) // max(1, int(os.environ.get("LOCAL_WORLD_SIZE", world))))
    t0 = time.perf_counter()
    fmm = SkelFMM(x, wl.kernel, tol, wl.leaf, kappa=wl.kappa, nrhs_max=nrhs, num_threads=threads,
                  device_build=args.build == "device", store_tiles=args.store_tiles, updown_tc=args.updown_tc)
    t_build = time.perf_counter() - t0
    # the tensor-core path covers the 3D kernels and 2D Laplace; 2D Helmholtz
    # (Bessel functions) runs on the CUDA cores
    prec = args.precision or ("fp32" if wl.kernel == "helmholtz2d" else "fp32_tc")
    tuning = None
    if args.tune == "auto" and not cplx and prec != "fp64":
        # outside the timed region, like the build: measure the variants on
        # this plan and keep the faster ones (results are unchanged)
        t0 = time.perf_counter()
        try:
            tuning = fmm.autotune(nrhs, allow_store=True)
            tuning["t_tune_s"] = time.perf_counter() - t0
        except Exception as e:                          # keep the untuned plan
            tuning = {"error": str(e)}
    if args.updown_shape is not None:
        from paper_2310_16668_gb300 import _lib
        _lib.check(_lib.load().skel_test_set_updown(fmm._h, args.updown_shape))
    info = fmm.info()
    pairs = info["pairs_direct"] + info["pairs_far"]

    if cplx:
        rdt = torch.complex128 if prec == "fp64" else torch.complex64
    else:
        rdt = torch.float64 if prec == "fp64" else torch.float32
    # column-major n x nrhs device buffers (each right-hand side contiguous)
    qc = torch.from_numpy(np.ascontiguousarray(q.T)).to(dev, rdt)
    uc = torch.empty_like(qc)
    stream = torch.cuda.current_stream(dev)

    def step():
        fmm.apply_into(qc, uc, nrhs, prec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    fmm.set_profiling(args.steps)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    phases = fmm.last_timings()
    fmm.set_profiling(0)
    if world > 1:
        dist.barrier()
        ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    value = whole_job_value(n, nrhs, world, ms_step)

    # errors against the oracle's direct sum on sampled targets: the first,
    # a middle and the last right-hand side (each 32-column pass of the
    # tensor-core path checked in its first, inner and last B-operand column)
    cols = sorted({0, min(17, nrhs - 1), nrhs - 1})
    u_cols = uc[cols].cpu().numpy().astype(np.complex128 if cplx else np.float64)
    sample = wl.make_sample() if n == wl0.n else np.sort(np.random.default_rng(5).choice(n, min(4096, n), replace=False))
    out = {}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle at the 4096 error-check targets for RHS 0 (timed: the
        # cpu_baseline), then at as many more random targets as fill about
        # 12 s of host time at the rate measured on the first part (the
        # kernels' costs differ by 30x); the other checked columns untimed
        q0 = np.ascontiguousarray(q[:, 0])
        ref, t_cpu, cores = oracle_direct_sample(wl.kernel, x, q0, sample, wl.kappa)
        n_more = int(min(n - len(sample), max(0.0, len(sample) / t_cpu * 12.0 - len(sample))))
        n_cpu = len(sample)
        if n_more > 0:
            rest = np.setdiff1d(np.arange(n), sample)
            more = np.sort(np.random.default_rng(11).choice(rest, n_more, replace=False))
            _, t_more, _ = oracle_direct_sample(wl.kernel, x, q0, more, wl.kappa)
            t_cpu += t_more
            n_cpu += n_more
        refs = {0: ref}
        for c in cols[1:]:
            refs[c] = oracle_direct_sample(wl.kernel, x, np.ascontiguousarray(q[:, c]), sample, wl.kappa)[0]
        errs, errs2 = {}, {}
        for i, c in enumerate(cols):
            d = u_cols[i][sample] - refs[c]
            errs[c] = float(np.abs(d).max() / np.abs(refs[c]).max())
            errs2[c] = float(np.linalg.norm(d) / np.linalg.norm(refs[c]))
        out["relerr"] = max(errs.values())
        out["relerr_l2"] = max(errs2.values())
        out["relerr_cols"] = {str(c): e for c, e in errs.items()}
        out["cpu_baseline"] = {"value": n_cpu / t_cpu / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"FP64 direct sum at {n_cpu} random targets x {n} sources, "
                                         f"RHS 0 ({t_cpu:.1f} s); value = targets / s"}
    else:
        ref = None

    # plain FP64 single-RHS apply on the same plan (the comparator)
    fp64 = None
    if not args.no_fp64 and prec != "fp64":
        q64 = torch.from_numpy(np.ascontiguousarray(q[:, :1].T)).to(dev, torch.complex128 if cplx else torch.float64)
        u64 = torch.empty_like(q64)
        k64 = max(1, min(args.steps, 5))
        for _ in range(2):
            fmm.apply_into(q64, u64, 1, "fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k64):
            fmm.apply_into(q64, u64, 1, "fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        fp64 = {"precision": "fp64", "nrhs": 1, "ms_per_step": ms64, "value": n / (ms64 * 1e-3) / 1e6,
                "unit": UNIT}
        if ref is not None:
            e64 = u64[0].cpu().numpy()[sample] - ref
            fp64["relerr"] = float(np.abs(e64).max() / np.abs(ref).max())
            fp64["relerr_l2"] = float(np.linalg.norm(e64) / np.linalg.norm(ref))

    # end to end through the C-ABI with pinned host buffers (H2D + apply + D2H per step)
    e2e = None
    if not args.no_e2e:
        qh = torch.from_numpy(np.ascontiguousarray(q.T)).to(rdt).pin_memory()
        uh = torch.empty_like(qh).pin_memory()
        fmm.apply_into(qh, uh, nrhs, prec, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        k = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(k):
            fmm.apply_into(qh, uh, nrhs, prec, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / k
        nb = qh.numel() * qh.element_size()
        if world > 1:
            dt = max_over_ranks(dt, dist, dev)
        e2e = {"value": whole_job_value(n, nrhs, world, dt * 1e3), "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb, "ms_per_step": dt * 1e3}

    if rank != 0:
        return 0
    roof = roofline(info, phases, clk, prec, pairs, wl.kernel, wl.name)
    _, peaks_kind = measured_peaks()
    metric = METRIC if args.workload == "laplace3d" else f"Mpts·RHS/s, {wl0.name} apply: {prec} vs plain FP64"
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": ("c128" if cplx else "f64") if prec == "fp64" else ("c64" if cplx else "f32"),
        "data": "synthetic",
        "config": {"workload": wl.name, "N": n, "nrhs": nrhs, "leaf": wl.leaf, "tol": tol, "precision": prec,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: operators + entry arrays "
                         f"{info['device_bytes'] / 1e9:.2f} GB resident",
                   "k_max": info["k_max"], "levels": info["n_levels"], "t_build_s": t_build,
                   "pairs_per_apply": pairs,
                   "updown": "tensor cores" if args.updown_tc and prec == "fp32_tc" else "CUDA cores",
                   "translations": ({1: "per-tile store", 2: "symmetric store"}.get(info["store_mode"], "kernel on the fly"))
                                   + (", chosen by skel_autotune" if tuning and "error" not in tuning else "")},
        "relerr": out.get("relerr"),
        "relerr_l2": out.get("relerr_l2"),
        "relerr_cols": out.get("relerr_cols"),
        "tuning": tuning,
        "build": {"where": args.build, "t_build_s": t_build, "t_tree_s": info["t_tree"], "t_skel_s": info["t_skel"],
                  "t_upload_s": info["t_upload"], "host_threads": threads,
                  "t_id_kernels_s": info["t_id_kernels"] if args.build == "device" else None,
                  "id_gflop": info["id_gflop"] if args.build == "device" else None,
                  "stored_tile_bytes": info["stored_tile_bytes"]},
        "comparator_fp64": fp64,
        "phases_ms_per_step": {k: v / phases["n_applies"] for k, v in phases.items()
                               if k not in ("launches", "n_applies", "main_launches")},
        "roofline": roof,
        "peaks_source": peaks_kind,
        "cpu_baseline": out.get("cpu_baseline"),
        "e2e": e2e,
        "gpu_launches": phases["launches"],
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                   "reasons": clk.get("reasons")},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "curves2d":
        return run_curves(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
