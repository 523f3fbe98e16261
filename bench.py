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


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32_tc", choices=["fp32_tc", "fp32", "fp64"])
    p.add_argument("--nrhs", type=int, default=32)
    p.add_argument("--tol", type=float, default=None)
    p.add_argument("--n", type=int, default=None, help="override N (testing only)")
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


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("skel_kernels.cuh", "apply.cu", "tc_kernels.cuh"):
        p = os.path.join(ROOT, "paper_2310_16668_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, precision: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    sha = kernel_source_sha()
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    pat = re.compile(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+kernel:\s*(\S+)\s+precision:\s*(\S+)\s+"
                     r"source_sha:\s*([0-9a-f]+)")
    for f in sorted(os.listdir(d)):
        if not f.endswith((".md", ".txt")):
            continue
        for m in pat.finditer(open(os.path.join(d, f)).read()):
            if m.group(2) == kernel and m.group(3) == precision and m.group(4) == sha:
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


def oracle_direct_sample(x, q0, targets):
    """The oracle's FP64 direct sum at `targets` (cpu_baseline leg)."""
    from oracle import direct
    t0 = time.perf_counter()
    u = direct.direct_sum("laplace3d", x, q0, targets=targets)
    return u, time.perf_counter() - t0, direct.num_threads()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import direct
    from paper_2310_16668_gb300 import workloads as W
    wl = W.LAPLACE3D_1M
    n = args.n or wl.n
    x = W.points_uniform(n, 3, wl.seed)
    q0 = W.charges_normal(n, 1, wl.seed + 1000)[:, 0]
    per_step = max(16, min(1024, int(1e9 // n)))       # ~1e9 pair evaluations per step
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        direct.direct_sum("laplace3d", x, q0, targets=rng.choice(n, per_step, replace=False))
    times = []
    for _ in range(args.steps):
        tg = rng.choice(n, per_step, replace=False)
        t0 = time.perf_counter()
        direct.direct_sum("laplace3d", x, q0, targets=tg)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    value = per_step * args.steps / T / 1e6
    cores = direct.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "N": n, "nrhs": 1, "sample_targets_per_step": per_step,
                   "method": "oracle FP64 direct sum (plain C, OpenMP), throughput extrapolated per target"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random targets x {n} sources x 1 RHS per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
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

    wl = W.LAPLACE3D_1M
    n = args.n or wl.n
    tol = args.tol or wl.tol
    nrhs = args.nrhs
    seed = replica_seed(wl.seed, rank)  # independent replica per rank
    x = W.points_uniform(n, 3, seed)
    q = W.charges_normal(n, nrhs, seed + 1000)
    threads = max(1, (os.cpu_count() or 1) // max(1, int(os.environ.get("LOCAL_WORLD_SIZE", world))))
    t0 = time.perf_counter()
    fmm = SkelFMM(x, wl.kernel, tol, wl.leaf, nrhs_max=nrhs, num_threads=threads)
    t_build = time.perf_counter() - t0
    info = fmm.info()
    pairs = info["pairs_direct"] + info["pairs_far"]

    prec = args.precision
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

    # errors against the oracle's direct sum on sampled targets (RHS 0)
    u_main = uc[0].double().cpu().numpy()
    sample = wl.make_sample() if n == wl.n else np.sort(np.random.default_rng(5).choice(n, min(4096, n), replace=False))
    out = {}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on 65,536 targets (about 10 s on 16 cores) that include the
        # 4096 error-check targets
        extra = np.random.default_rng(11).choice(n, min(n, 65536), replace=False)
        big = np.union1d(sample, extra)
        ref_big, t_cpu, cores = oracle_direct_sample(x, q[:, 0], big)
        ref = ref_big[np.searchsorted(big, sample)]
        scale = np.abs(ref).max()
        out["relerr"] = float(np.abs(u_main[sample] - ref).max() / scale)
        out["cpu_baseline"] = {"value": len(big) / t_cpu / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"FP64 direct sum at {len(big)} random targets x {n} sources, "
                                         f"RHS 0 ({t_cpu:.1f} s); value = targets / s"}
    else:
        ref = None

    # plain FP64 single-RHS apply on the same plan (the comparator)
    fp64 = None
    if not args.no_fp64 and prec != "fp64":
        q64 = torch.from_numpy(np.ascontiguousarray(q[:, :1].T)).to(dev, torch.float64)
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
            fp64["relerr"] = float(np.abs(u64[0].cpu().numpy()[sample] - ref).max() / np.abs(ref).max())

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
    # roofline of the dominant kernel, the main translation kernel (kernel
    # evaluations; MUFU rsqrt-bound): on the tensor-core path one launch per
    # 32 right-hand sides over the pairs of the tensor-core items, timed by
    # the plan's own events on the launching stream (the CUDA-core launch for
    # the small non-leaf boxes is outside that span)
    if prec == "fp32_tc":
        kname, units = "tc_near_kernel", info["pairs_tc"]
        unit_note = "skel_info pairs_tc: kept kernel evaluations of the tensor-core items"
    else:
        kname, units = "near_kernel", pairs
        unit_note = "skel_info pairs_direct + pairs_far"
    n_near = phases["main_launches"] / phases["n_applies"]
    near_ms_per_launch = phases["main_near"] / phases["main_launches"]
    achieved = units / (near_ms_per_launch * 1e-3) / 1e9
    sm_mhz = clk.get("sm_mhz") or 2070.0
    peak = SM_COUNT * MUFU_PER_SM_CLK * sm_mhz * 1e6 / 1e9
    peaks, peaks_kind = measured_peaks()
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
            "frac": achieved / peak, "traffic": ncu_traffic(kname, prec),
            "peak_basis": f"{SM_COUNT} SMs x {MUFU_PER_SM_CLK} MUFU rsqrt/clk x median SM clock under load "
                          f"({sm_mhz:.0f} MHz)",
            "per_launch_ms": near_ms_per_launch, "launches_per_step": n_near,
            "algorithmic_units": f"{units} kernel evaluations per launch ({unit_note})"}
    if prec == "fp32_tc":
        # the same launch against the tensor pipe: algorithmic 2 flops per
        # evaluation and right-hand side (32 per launch); the pipe issues 3
        # TF32 products (hi.hi + hi.lo + lo.hi) over full 128 x 32 tiles
        tc_tflops = units * 2 * 32 / (near_ms_per_launch * 1e-3) / 1e12
        issued = info["n_tc_tiles"] * 128 * 32 * 32 * 2 * 3 / (near_ms_per_launch * 1e-3) / 1e12
        tf32_peak = peaks["bf16_tflops"] * 0.5
        roof["tensor"] = {"achieved": tc_tflops, "peak": tf32_peak, "unit": "TFLOP/s", "frac": tc_tflops / tf32_peak,
                          "issued_tflops": issued,
                          "peak_basis": f"TF32 = 0.5 x {peaks_kind} bf16 burst ({peaks['bf16_tflops']} TFLOP/s)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": wl.name, "N": n, "nrhs": nrhs, "leaf": wl.leaf, "tol": tol, "precision": prec,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: operators + entry arrays "
                         f"{info['device_bytes'] / 1e9:.2f} GB resident",
                   "k_max": info["k_max"], "levels": info["n_levels"], "t_build_s": t_build,
                   "pairs_per_apply": pairs},
        "relerr": out.get("relerr"),
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
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
