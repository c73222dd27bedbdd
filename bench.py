"""Benchmark of the J-VIE operator application on one GB300 (or N replicas).

Workload: the truncated Si strip guide, 600 x 23 x 11 voxels (h = 20 nm,
eps_core = 12.11 in eps_bg = 2.085, quadratic absorber over the last 4 um),
complex64 operator application y = w - M (N w) through the C ABI.

A step is one operator application on a fresh input vector.  Inputs cycle
through a pool whose inputs and outputs together exceed the 129 MB L2, so no
step starts with its vector cached.  The timed region is bracketed by a
barrier and a device synchronisation on both sides and timed with CUDA events
on the launching stream; rank 0 prints one JSON line with the maximum time
over ranks.  Multi-GPU runs are independent replicas (weak scaling): the
operator does not shard.

`--impl reference` times the FP64 CPU oracle (the baseline of this project)
on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VIE matvecs/s & time-to-1e-6 residual; mixed+learned vs plain FP64, 1 GB300"
UNIT = "matvecs/s"
L2_BYTES = 129 * 1024 * 1024
WORKLOAD = ("Si strip waveguide 600x23x11 voxels, h=20nm, eps_core=12.11, eps_bg=2.085, "
            "quadratic absorber over the last 4um (R_rt=1e-10), complex64 operator application")


FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # FP32 FMA lanes x 2 flop x max SM clock


def operator_flops(grid, m, y_first: bool = False) -> float:
    """Algorithmic FP32 flops of one operator application: 5 L log2 L per
    complex FFT of length L on the lines that carry data (x: the 3 ny nz
    non-zero lines, forward and inverse; per kx plane: 3 ny z-lines and 3 Mz
    y-lines, forward and inverse, or 3 nz y-lines and 3 My z-lines when y is
    transformed first) plus 72 flops per spectral cell for the symmetric 3x3
    complex multiply."""
    nx, ny, nz = grid
    Mx, My, Mz = m
    f = lambda L: 5.0 * L * math.log2(L) if L > 1 else 0.0
    x_part = 3 * ny * nz * 2 * f(Mx)
    if y_first:
        plane = 3 * nz * 2 * f(My) + 3 * My * 2 * f(Mz) + 72.0 * My * Mz
    else:
        plane = 3 * ny * 2 * f(Mz) + 3 * Mz * 2 * f(My) + 72.0 * My * Mz
    return x_part + Mx * plane


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def _bf16_peak():
    """Dense BF16 tensor peak in TFLOP/s (burst), measured if available."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops" in d:
            return d["bf16_tflops"], "measured"
    return 1900.0, "fallback"


NET_LAYERS = [(8, 32, 0), (32, 32, 1), (32, 32, 2), (32, 32, 3), (32, 32, 2), (32, 32, 1), (32, 32, 0), (32, 6, 0)]


def net_flops(grid) -> float:
    """Algorithmic tensor flops of one network application: 2 x 27 x ci x co
    per voxel of each convolution's level (levels halve nx and ny, ceil)."""
    nx, ny, nz = grid
    vox = []
    for _ in range(4):
        vox.append(nx * ny * nz)
        nx, ny = (nx + 1) // 2, (ny + 1) // 2
    return sum(2.0 * 27 * ci * co * vox[lvl] for ci, co, lvl in NET_LAYERS)


def net_section(plan, grid, reps=50):
    """Inference cost of the learned preconditioner on the benchmark grid
    (random parameters in every layer; the cost does not depend on them)."""
    import torch

    from paper_1803_06237_gb300 import vie
    n = vie.vie_net_param_count()
    rng = np.random.default_rng(3)
    net = vie.vie_net_create(rng.standard_normal(n).astype(np.float32) * 0.05)
    v = torch.randn(3 * plan.n_vox, dtype=torch.complex64, device="cuda")
    z = torch.empty_like(v)
    stream = torch.cuda.current_stream()
    for _ in range(5):
        vie.vie_net_apply(net, plan, v, z, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        vie.vie_net_apply(net, plan, v, z, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    net.close()
    flops = net_flops(grid)
    peak, kind = _bf16_peak()
    tf = flops / (ms * 1e-3) / 1e12
    return {"ms_per_apply": ms, "algorithmic_flops": flops,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "peak_source": kind + " dense bf16 (burst)"},
            "launches_per_apply": 10,
            "note": "|v|^2, input packing and 8 tcgen05 convolutions (pooling, upsample-add and the output "
                    "step fused into their epilogues); the convolutions' 3x3x3 flops only"}


class ClockSampler:
    """Samples nvidia-smi during the timed region (every 200 ms)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

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
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def clock_snapshot(index: int) -> dict:
    """One nvidia-smi read of the SM clock, its maximum and the throttle
    reasons (before and after the timed region, which can be shorter than the
    sampler's 200 ms period)."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), f"--query-gpu={ClockSampler.FIELDS}",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20).stdout
    except (OSError, subprocess.TimeoutExpired):
        return {}
    parts = [x.strip() for x in out.strip().split(",")]
    if len(parts) < 8:
        return {}
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        return {"sm_mhz": float(parts[0]), "sm_max_mhz": float(parts[1]), "power_w": float(parts[2]),
                "reasons": [n for n, v in zip(names, parts[4:8]) if v.lower().startswith("active")]}
    except ValueError:
        return {}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The slowest rank's time (every rank gets it); `device` is where the
    process group's collectives run ("cuda" for NCCL, "cpu" for gloo)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, ms: float) -> float:
    """Units per second for the whole job: every rank did `steps` units in
    at most `ms` milliseconds (weak scaling)."""
    return world * steps / (ms / 1e3)


def captured_traffic(info: dict, path: str | None = None):
    """(x_passes, DRAM bytes per guide operator application) from the
    committed ncu capture, the bytes only when the plan runs the x-pass
    kernels that capture measured (else None).  The default codes (0) are,
    for the guide's 759 lines, the three-factor forward and the four-step
    inverse pass, both with five lines per block."""
    x_passes = [info["x_lines_per_block"] or -5, info["x_lines_per_block_inverse"] or 5]
    tp = path or os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tj = json.load(open(tp))
    except (OSError, ValueError):
        return x_passes, None
    if tj.get("x_passes") != x_passes:
        return x_passes, None
    return x_passes, tj.get("matvec_c64_waveguide_bytes")


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    from paper_1803_06237_gb300 import build, vie, workloads

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build_library()
    vie.load()

    wl = workloads.waveguide()
    ab = wl.absorbers[0]
    e2 = vie.vie_eps2_from_round_trip(ab.r_rt, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
    absorbers = [dict(x0=ab.x0, length=ab.length, degree=ab.degree, eps2_max=e2)]
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg,
                               vie.VIE_PLAN_AUTOTUNE if args.autotune else vie.VIE_PLAN_DEFAULT)
    vie.vie_set_permittivity(plan, wl.eps, absorbers)
    info = plan.info()

    n3 = 3 * wl.n_voxels
    vec_bytes = n3 * 8
    pool = max(2, int(np.ceil(1.5 * L2_BYTES / (2 * vec_bytes))))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234 + rank)
    xs = torch.randn((pool, n3), dtype=torch.complex64, device="cuda", generator=gen)
    ys = torch.empty_like(xs)
    stream = torch.cuda.current_stream()

    for i in range(args.warmup):
        vie.vie_matvec(plan, xs[i % pool], ys[i % pool], stream)
    torch.cuda.synchronize()

    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.25)                      # the sampler's first line
    clk_before = clock_snapshot(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(K):
        vie.vie_matvec(plan, xs[i % pool], ys[i % pool], stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk_after = clock_snapshot(local)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    clk["before"] = clk_before
    clk["after"] = clk_after
    if clk.get("sm_mhz") is None:
        reads = [c["sm_mhz"] for c in (clk_before, clk_after) if c.get("sm_mhz")]
        clk["sm_mhz"] = statistics.median(reads) if reads else None
        clk["sm_max_mhz"] = max([c["sm_max_mhz"] for c in (clk_before, clk_after) if c.get("sm_max_mhz")],
                                default=None)
        clk["reasons"] = sorted(set(clk.get("reasons", [])) | set(clk_before.get("reasons", []))
                                | set(clk_after.get("reasons", [])))
        clk["source"] = "nvidia-smi reads just before and after the timed region (shorter than the 200 ms sampler)"
    ms = max_over_ranks(ev[0].elapsed_time(ev[1]), world, "cuda")
    per_step_ms = ms / K
    value = whole_job_rate(world, K, ms)

    # end to end through the public API with host buffers (pinned), copies timed
    Ke = min(K, args.e2e_steps)
    hx = torch.randn((n3,), dtype=torch.complex64).pin_memory()
    hy = torch.empty((n3,), dtype=torch.complex64).pin_memory()
    dx = torch.empty((n3,), dtype=torch.complex64, device="cuda")
    dy = torch.empty_like(dx)
    for _ in range(3):
        dx.copy_(hx, non_blocking=True)
        vie.vie_matvec(plan, dx, dy, stream)
        hy.copy_(dy, non_blocking=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        dx.copy_(hx, non_blocking=True)
        vie.vie_matvec(plan, dx, dy, stream)
        hy.copy_(dy, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    e2e_value = whole_job_rate(world, Ke, e2e_ms)

    # spread of the per-application time, outside the timed region: 20 bursts
    # of ten applications from the same input pool, each burst between two
    # CUDA events on the launching stream; median and 10th / 90th percentiles
    try:
        nb, bl = 20, 10
        bev = [torch.cuda.Event(enable_timing=True) for _ in range(nb + 1)]
        bev[0].record(stream)
        for b_ in range(nb):
            for i in range(bl):
                j = b_ * bl + i
                vie.vie_matvec(plan, xs[j % pool], ys[j % pool], stream)
            bev[b_ + 1].record(stream)
        torch.cuda.synchronize()
        per_us = [bev[b_].elapsed_time(bev[b_ + 1]) * 1e3 / bl for b_ in range(nb)]
        p10, p50, p90 = (float(v) for v in np.percentile(per_us, [10, 50, 90]))
        spread = {"median": p50, "p10": p10, "p90": p90, "unit": "us per application", "bursts": nb,
                  "applications_per_burst": bl}
    except Exception as exc:                  # reported, never fatal to the line
        spread = {"error": str(exc)[:200]}

    # measured FP32 / FP64 FMA rates (the ALU roofline), outside the timed region
    fp32_peak = vie.vie_probe_fma_tflops(vie.VIE_C64)
    fp64_peak = vie.vie_probe_fma_tflops(vie.VIE_C128)

    # roofline of the operator application (its three launches are the unit)
    nx, ny, nz = wl.grid
    Mx, My, Mz = info["m"]
    Kx, Ky, Kz = (m // 2 + 1 for m in info["m"])
    s = 8
    alg_bytes = (3 * wl.n_voxels * 2 + wl.n_voxels) * s + 6 * Kx * Ky * Kz * s
    alg_flops = operator_flops(wl.grid, info["m"])
    t_s = per_step_ms * 1e-3
    hbm_peak, peak_kind = _peaks()
    alu_peak = fp32_peak
    achieved_tf = alg_flops / t_s / 1e12
    x_passes, traffic = captured_traffic(info)
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / alu_peak, "traffic": traffic,
                "kernel": "complex64 operator application (passes A, B, C)", "x_passes": x_passes,
                "algorithmic_flops_per_launch": alg_flops, "algorithmic_bytes_per_launch": alg_bytes,
                "peak_source": "measured FP32 FMA throughput (vie_probe_fma_tflops); nominal %.1f = "
                               "152 SMs x 128 lanes x 2 flop x 2.07 GHz" % FP32_TFLOPS,
                "hbm": {"achieved": alg_bytes / t_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": alg_bytes / t_s / 1e9 / hbm_peak, "peak_source": peak_kind}}
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": per_step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(wl.grid), "circulant": list(info["m"]),
                   "autotune": ({"candidates": info["tune_candidates"], "ms": round(info["tune_ms"], 1),
                                 "x_lines_per_block": info["x_lines_per_block"],
                                 "x_lines_per_block_inverse": info["x_lines_per_block_inverse"]}
                                if args.autotune else None),
                   "input_pool_vectors": pool, "l2": f"inputs+outputs cycle through {2 * pool * vec_bytes / 2**20:.0f} MiB > 129 MB L2",
                   "parallelism": f"{world} independent replicas"},
        "step_time_spread": spread,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": vec_bytes, "d2h_bytes_per_step": vec_bytes,
                "steps": Ke},
        "gpu_launches": 3 * K,
        "roofline": roofline,
        "clocks": clk,
        "setup_ms": info["setup_ms"],
        "alu_peaks_measured": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak,
                               "how": "FMA chains on every SM, CUDA events (vie_probe_fma_tflops)"},
        "c128_operator": c128_section(plan, wl, info, fp64_peak, alg_flops),
        "cufft_reference": cufft_reference(wl, info, per_step_ms),
    }
    if not args.no_net:
        result["net_inference"] = net_section(plan, wl.grid)
    if not args.no_solve:
        result["time_to_1e-6"] = solve_section(plan, wl, absorbers, args)
    if not args.no_batch:
        result["batch48"] = batch_section(args)
    if args.microring:
        result["microring"] = microring_section(args, fp32_peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def c128_section(plan, wl, info, fp64_peak, alg_flops, reps=100):
    """The complex128 operator (the refinement's outer residual) on the same
    guide: applications per second, against the measured FP64 FMA rate (same
    algorithmic flop count as complex64) and the HBM roofline."""
    import torch

    from paper_1803_06237_gb300 import vie
    n3 = 3 * wl.n_voxels
    pool = max(2, int(np.ceil(1.5 * L2_BYTES / (2 * n3 * 16))))
    xs = torch.randn((pool, n3), dtype=torch.complex128, device="cuda")
    ys = torch.empty_like(xs)
    stream = torch.cuda.current_stream()
    for i in range(3):
        vie.vie_matvec(plan, xs[i % pool], ys[i % pool], stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        vie.vie_matvec(plan, xs[i % pool], ys[i % pool], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    Kx, Ky, Kz = (m // 2 + 1 for m in info["m"])
    alg_bytes = (3 * wl.n_voxels * 2 + wl.n_voxels) * 16 + 6 * Kx * Ky * Kz * 16
    hbm_peak, kind = _peaks()
    tf = alg_flops / (ms * 1e-3) / 1e12
    return {"ms_per_matvec": ms, "matvecs_per_s": 1e3 / ms, "input_pool_vectors": pool,
            "alu": {"bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": tf / fp64_peak,
                    "peak_source": "measured FP64 FMA throughput"},
            "hbm": {"achieved": alg_bytes / ms / 1e6, "peak": hbm_peak, "unit": "GB/s",
                    "frac": alg_bytes / ms / 1e6 / hbm_peak, "algorithmic_bytes": alg_bytes, "peak_source": kind}}


def cufft_reference(wl, info, our_ms, reps=50):
    """Reference point only (not the product path): the same operator shape
    written with PyTorch's FFTs (cuFFT) and element-wise ops: pad the three
    components into the circulant embedding, 3-D forward FFT, the symmetric
    3x3 spectral multiply with six full spectra (random values: timing
    only), inverse FFT, crop, y = x - M (N x).  Complex64, CUDA events."""
    import torch
    Mx, My, Mz = info["m"]
    nx, ny, nz = wl.grid
    g = torch.Generator(device="cuda").manual_seed(7)
    G = torch.randn((6, Mz, My, Mx), dtype=torch.complex64, device="cuda", generator=g)
    Mc = torch.randn((nz, ny, nx), dtype=torch.complex64, device="cuda", generator=g)
    x = torch.randn((3, nz, ny, nx), dtype=torch.complex64, device="cuda", generator=g)
    pad = torch.zeros((3, Mz, My, Mx), dtype=torch.complex64, device="cuda")

    def apply(x):
        pad.zero_()
        pad[:, :nz, :ny, :nx] = x
        X = torch.fft.fftn(pad, dim=(1, 2, 3))
        Y = torch.stack([G[0] * X[0] + G[3] * X[1] + G[4] * X[2],
                         G[3] * X[0] + G[1] * X[1] + G[5] * X[2],
                         G[4] * X[0] + G[5] * X[1] + G[2] * X[2]])
        y = torch.fft.ifftn(Y, dim=(1, 2, 3))[:, :nz, :ny, :nx]
        return x - Mc * y

    for _ in range(3):
        apply(x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        apply(x)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"ms_per_matvec": ms, "matvecs_per_s": 1e3 / ms, "ours_over_cufft_speedup": ms / our_ms,
            "what": "torch.fft.fftn/ifftn (cuFFT) on the 3 x %d x %d x %d embedding + PyTorch element-wise "
                    "multiply, crop and contrast; random spectra; reference point only" % (Mx, My, Mz)}


def _timed_solve(plan, b, mode, restart, use_pc, keep=None):
    import torch

    from paper_1803_06237_gb300 import vie
    x = torch.zeros_like(b)
    if keep is not None:
        keep.append(x)
    torch.cuda.synchronize()
    t = time.perf_counter()
    info = vie.vie_solve(plan, b, x, 1e-6, mode=mode, restart=restart, use_preconditioner=use_pc,
                         raise_on_not_converged=False)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t) * 1e3
    return {"ms": wall, "device_ms": info["time_ms"], "iterations": info["iterations"], "cycles": info["outer"],
            "matvecs_c128": info["matvecs64"], "matvecs_c64": info["matvecs32"], "converged": info["converged"],
            "true_residual": info["residual"], "preconditioner_dropped": info["fallback"], "restart": restart,
            "graph_cycles": info["graph_cycles"], "reorth_steps": info["reorth_steps"]}


def microring_section(args, fp32_peak, reps=40, reps64=8):
    """Operator on the 800 x 600 x 11 ring resonator (circulant 1600 x 1200 x
    24, pass B on CTA clusters): plan setup, complex64 and complex128
    applications timed with CUDA events on two input/output pairs of 127 MB
    each (larger than L2)."""
    import torch

    from paper_1803_06237_gb300 import vie, workloads
    wl = workloads.microring()
    absorbers = []
    for ab in wl.absorbers:
        e2 = vie.vie_eps2_from_round_trip(ab.r_rt, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
        absorbers.append(dict(x0=ab.x0, length=ab.length, degree=ab.degree, direction=ab.direction, eps2_max=e2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    setup_host_ms = (time.perf_counter() - t0) * 1e3
    vie.vie_set_permittivity(plan, wl.eps, absorbers)
    info = plan.info()
    n3 = 3 * wl.n_voxels
    stream = torch.cuda.current_stream()
    out = {"grid": list(wl.grid), "circulant": list(info["m"]), "setup_ms": round(setup_host_ms, 1),
           "device_bytes": info["device_bytes"]}
    for dtype, name, r in ((torch.complex64, "c64", reps), (torch.complex128, "c128", reps64)):
        xs = torch.randn((2, n3), dtype=dtype, device="cuda")
        ys = torch.empty_like(xs)
        for i in range(3):
            vie.vie_matvec(plan, xs[i % 2], ys[i % 2], stream)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for i in range(r):
            vie.vie_matvec(plan, xs[i % 2], ys[i % 2], stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / r
        es = xs.element_size()
        Kx, Ky, Kz = (m // 2 + 1 for m in info["m"])
        alg_bytes = (3 * wl.n_voxels * 2 + wl.n_voxels) * es + 6 * Kx * Ky * Kz * es
        hbm_peak, peak_kind = _peaks()
        entry = {"ms_per_matvec": ms, "matvecs_per_s": 1e3 / ms,
                 "hbm": {"algorithmic_bytes": alg_bytes, "achieved": alg_bytes / ms / 1e6, "peak": hbm_peak,
                         "unit": "GB/s", "frac": alg_bytes / ms / 1e6 / hbm_peak, "peak_source": peak_kind}}
        if dtype == torch.complex64:
            fl = operator_flops(wl.grid, info["m"], y_first=True)
            entry["alu"] = {"algorithmic_flops": fl, "achieved": fl / ms / 1e9, "peak": fp32_peak,
                            "unit": "TFLOP/s", "frac": fl / ms / 1e9 / fp32_peak,
                            "peak_source": "measured FP32 FMA throughput"}
        out[name] = entry
        del xs, ys
    plan.close()
    return out


def solve_section(plan, wl, absorbers, args):
    """Time to a true FP64 relative residual of 1e-6 on the benchmark guide
    (Gaussian sheet source): plain complex128 GMRES, mixed precision, and
    mixed precision with the learned preconditioner (trained first, outside
    the timed solves, on pairs from plain solves of random strips and bends)."""
    import torch

    from paper_1803_06237_gb300 import learned, vie
    src = torch.from_numpy(np.ascontiguousarray(wl.src.ravel())).cuda()
    b = torch.empty_like(src)
    vie.vie_rhs_from_source(plan, src, b)
    _timed_solve(plan, b, vie.VIE_SOLVE_MIXED, args.restart_mixed, False)      # warm-up (workspaces)
    sols = {}
    out = {}
    for name, mode, restart in (("fp64", vie.VIE_SOLVE_FP64, args.restart_fp64),
                                ("mixed", vie.VIE_SOLVE_MIXED, args.restart_mixed)):
        keep = []
        out[name] = _timed_solve(plan, b, mode, restart, False, keep)
        sols[name] = keep[0]
    if args.train_steps > 0:
        t0 = time.perf_counter()
        pairs = learned.make_pairs(range(args.train_problems), grid=(160, 40, 11), restart=20, cycles=10)
        t1 = time.perf_counter()
        net = vie.vie_net_create(seed=1)
        losses = learned.train(net, pairs, steps=args.train_steps, lr=1e-3, batch=4)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        v = torch.randn(b.numel(), dtype=torch.complex64, device="cuda")
        z = torch.empty_like(v)
        for _ in range(3):
            vie.vie_net_apply(net, plan, v, z)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(20):
            vie.vie_net_apply(net, plan, v, z)
        ev1.record()
        torch.cuda.synchronize()
        net_ms = ev0.elapsed_time(ev1) / 20
        vie.vie_set_preconditioner_net(plan, net)
        _timed_solve(plan, b, vie.VIE_SOLVE_MIXED, args.restart_mixed, True)   # warm-up
        keep = []
        out["mixed_learned"] = _timed_solve(plan, b, vie.VIE_SOLVE_MIXED, args.restart_mixed, True, keep)
        sols["mixed_learned"] = keep[0]
        out["training"] = {"pairs": len(pairs), "problems": args.train_problems, "steps": args.train_steps,
                           "identity_loss": learned.identity_loss(pairs),
                           "pair_generation_s": t1 - t0, "train_s": t2 - t1,
                           "loss_first20": float(np.mean(losses[:20])), "loss_last20": float(np.mean(losses[-20:])),
                           "net_apply_ms": net_ms, "precision": "bf16 tensor cores, fp32 accumulation"}
        vie.vie_set_preconditioner_net(plan, None)
    if args.circulant:
        out["circulant"] = circulant_section(plan, b, args)
        out["mixed_circulant"] = out["circulant"].pop("solve")
        sols["mixed_circulant"] = out["circulant"].pop("x")
        out["circulant_fp16"] = circulant_section(plan, b, args, fp16=True)
        out["mixed_circulant_fp16"] = out["circulant_fp16"].pop("solve")
        sols["mixed_circulant_fp16"] = out["circulant_fp16"].pop("x")
        out["accuracy"] = accuracy_section(plan, wl, b, sols, args)
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    if "mixed_learned" in out:
        out["speedup_mixed_learned_vs_fp64"] = out["fp64"]["ms"] / out["mixed_learned"]["ms"]
    if "mixed_circulant" in out:
        out["speedup_mixed_circulant_vs_fp64"] = out["fp64"]["ms"] / out["mixed_circulant"]["ms"]
        out["speedup_mixed_circulant_fp16_vs_fp64"] = out["fp64"]["ms"] / out["mixed_circulant_fp16"]["ms"]
    return out


def circulant_section(plan, b, args, reps=20, fp16=False):
    """The block-circulant preconditioner (Sec. 5.4) on the benchmark guide:
    setup (blocks, DFT along x, batched LU) timed on the host clock, the
    application timed with CUDA events against the HBM roofline (it streams
    the nx (3 ny nz)^2 complex64 factors once), and the preconditioned mixed
    solve to 1e-6."""
    import torch

    from paper_1803_06237_gb300 import vie
    flags = vie.VIE_CIRC_FP16_FACTORS if fp16 else vie.VIE_CIRC_DEFAULT
    # the first build in a process also pays one-time set-up (module loading,
    # first launches): timed separately, then a warm build is timed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vie.vie_circulant_create(plan, flags).close()
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    c = vie.vie_circulant_create(plan, flags)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    info = vie.vie_circulant_info(c)
    v = torch.randn(b.numel(), dtype=torch.complex64, device="cuda")
    z = torch.empty_like(v)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        vie.vie_circulant_apply(c, v, z, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        vie.vie_circulant_apply(c, v, z, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nx, ny, nz = plan.n
    R = 3 * ny * nz
    factor_bytes = nx * R * R * (4 if fp16 else 8)
    hbm_peak, kind = _peaks()
    achieved = factor_bytes / (ms * 1e-3) / 1e9
    vie.vie_set_circulant_preconditioner(plan, c)
    _timed_solve(plan, b, vie.VIE_SOLVE_MIXED, args.restart_mixed, True)      # warm-up
    keep = []
    solve = _timed_solve(plan, b, vie.VIE_SOLVE_MIXED, args.restart_mixed, True, keep)
    vie.vie_set_circulant_preconditioner(plan, None)
    c.close()
    return {"setup_ms": setup_ms, "setup_first_in_process_ms": first_ms, "build_ms_library": info["build_ms"],
            "device_bytes": info["device_bytes"],
            "apply_ms": ms,
            "apply_roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                               "frac": achieved / hbm_peak, "peak_source": kind,
                               "algorithmic_bytes": factor_bytes,
                               "note": "LU factors of the nx blocks (%s) read once per application"
                                       % ("complex half" if fp16 else "complex64")},
            "solve": solve, "x": keep[0]}


def accuracy_section(plan, wl, b, sols, args):
    """Accuracy of the timed solves (Sec. 5.1 R, Sec. 3 fields): the field
    error of each timed solution against a tight solve of the same guide
    (complex128 flexible GMRES with the block-circulant preconditioner to a
    true residual of 1e-10), and the reflection coefficient of the 4 um
    absorber: R = sum |E_ref - E|^2 / sum |E_ref|^2 on the axis before the
    absorber, E_ref from the same guide with a 12 um absorber (same R_rt)."""
    import torch

    from paper_1803_06237_gb300 import vie, workloads

    def tight(p, rhs, tol):
        c = vie.vie_circulant_create(p, vie.VIE_CIRC_DEFAULT)
        vie.vie_set_circulant_preconditioner(p, c)
        x = torch.zeros_like(rhs)
        inf = vie.vie_solve(p, rhs, x, tol, mode=vie.VIE_SOLVE_FP64, restart=args.restart_mixed,
                            use_preconditioner=True, raise_on_not_converged=False)
        vie.vie_set_circulant_preconditioner(p, None)
        c.close()
        return x, inf

    x_ref, inf = tight(plan, b, 1e-10)
    out = {"reference_solve": {"mode": "complex128 flexible GMRES + block-circulant", "true_residual": inf["residual"],
                               "converged": inf["converged"]},
           "field_rel_l2": {k: float((torch.linalg.vector_norm(v - x_ref) / torch.linalg.vector_norm(x_ref)).item())
                            for k, v in sols.items()}}
    body = int(round(wl.absorbers[0].x0))
    L_ref = 12.0
    wl2 = workloads.waveguide(nx=body + int(round(L_ref / wl.h_um)), absorber_len_um=L_ref)
    ab2 = wl2.absorbers[0]
    e2 = vie.vie_eps2_from_round_trip(ab2.r_rt, ab2.degree, ab2.length * wl2.h_um, wl2.k0_per_um, wl2.eps_core)
    plan2 = vie.vie_plan_create(wl2.grid, wl2.h_um, wl2.k0_per_um, wl2.eps_bg)
    vie.vie_set_permittivity(plan2, wl2.eps, [dict(x0=ab2.x0, length=ab2.length, degree=ab2.degree, eps2_max=e2)])
    src2 = torch.from_numpy(np.ascontiguousarray(wl2.src.ravel())).cuda()
    b2 = torch.empty_like(src2)
    vie.vie_rhs_from_source(plan2, src2, b2)
    x2, inf2 = tight(plan2, b2, 1e-10)
    e_ref = vie.vie_axis_field(plan2, x2, body)
    R = {"tight": vie.vie_reflection(e_ref, vie.vie_axis_field(plan, x_ref, body))}
    for k, v in sols.items():
        R[k] = vie.vie_reflection(e_ref, vie.vie_axis_field(plan, v, body))
    plan2.close()
    out["reflection"] = {"R": R, "absorber_um": wl.absorbers[0].length * wl.h_um, "reference_absorber_um": L_ref,
                         "axis_voxels": body, "reference_true_residual": inf2["residual"],
                         "note": "R of each timed solve's field and of the tight solve"}
    return out


def batch_section(args):
    """The 48 uneven guides solved together to 1e-6 (mixed precision), and
    the grouped operator on all 48 (complex64 applications per second)."""
    import torch

    from paper_1803_06237_gb300 import learned, vie, workloads
    wls = workloads.batch48()
    plans, bs, base = [], [], {}
    for wl in wls:
        plan, b = learned.setup_problem(wl, base.get(wl.grid))
        base.setdefault(wl.grid, plan)
        plans.append(plan)
        bs.append(b)
    xs = [torch.zeros_like(b) for b in bs]
    vie.vie_solve_batch(plans, bs, xs, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=args.restart_mixed,
                        raise_on_not_converged=False)                                      # warm-up
    xs = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    t = time.perf_counter()
    st, infos = vie.vie_solve_batch(plans, bs, xs, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=args.restart_mixed,
                                    raise_on_not_converged=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    # the same 48 solves as one graph launch (device-side decisions between
    # cycles and refinement steps)
    xs = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    t = time.perf_counter()
    st_r, infos_r = vie.vie_solve_batch(plans, bs, xs, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=args.restart_mixed,
                                        raise_on_not_converged=False, resident=True)
    torch.cuda.synchronize()
    wall_r = time.perf_counter() - t
    resident = {"solve_s": wall_r, "device_s": infos_r[0]["time_ms"] / 1e3, "status": st_r,
                "converged": sum(1 for i in infos_r if i["converged"]),
                "max_true_residual": max(i["residual"] for i in infos_r),
                "iterations_total": sum(i["iterations"] for i in infos_r),
                "note": "the whole solve as one CUDA graph launch (conditional WHILE/IF nodes)"}
    # the same 48 solves with a block-circulant preconditioner per guide
    # (complex-half factors), setup timed separately
    torch.cuda.synchronize()
    t = time.perf_counter()
    circs = [vie.vie_circulant_create(p, vie.VIE_CIRC_FP16_FACTORS) for p in plans]
    for p, c in zip(plans, circs):
        vie.vie_set_circulant_preconditioner(p, c)
    torch.cuda.synchronize()
    circ_setup = time.perf_counter() - t
    xs = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    t = time.perf_counter()
    st_c, infos_c = vie.vie_solve_batch(plans, bs, xs, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=args.restart_mixed,
                                        use_preconditioner=True, raise_on_not_converged=False)
    torch.cuda.synchronize()
    wall_c = time.perf_counter() - t
    for p in plans:
        vie.vie_set_circulant_preconditioner(p, None)
    for c in circs:
        c.close()
    del circs
    v64 = [torch.randn(3 * p.n_vox, dtype=torch.complex64, device="cuda") for p in plans]
    y64 = [torch.empty_like(v) for v in v64]
    for _ in range(3):
        vie.vie_matvec_batch(plans, v64, y64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 50
    e0.record()
    for _ in range(reps):
        vie.vie_matvec_batch(plans, v64, y64)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    vox = sum(p.n_vox for p in plans)
    return {"problems": len(plans), "voxels": vox, "solve_s": wall, "status": st,
            "converged": sum(1 for i in infos if i["converged"]),
            "max_true_residual": max(i["residual"] for i in infos),
            "iterations_total": sum(i["iterations"] for i in infos),
            "grouped_matvec_ms": ms, "grouped_matvecs_per_s": len(plans) * 1e3 / ms,
            "resident": resident,
            "circulant": {"setup_s": circ_setup, "solve_s": wall_c, "status": st_c,
                          "converged": sum(1 for i in infos_c if i["converged"]),
                          "max_true_residual": max(i["residual"] for i in infos_c),
                          "iterations_total": sum(i["iterations"] for i in infos_c),
                          "preconditioner_dropped": sum(1 for i in infos_c if i["fallback"]),
                          "factors": "complex half"},
            "note": "solve_s covers all 48 problems in one vie_solve_batch call"}


def _oracle_setup():
    """The oracle's FFT matvec (scipy, complex128) on the full guide with a
    synthetic spectrum of the right shape (spectrum values do not change the
    cost): returns a callable doing one application."""
    from oracle import operator as op
    from paper_1803_06237_gb300 import workloads

    wl = workloads.waveguide()
    nx, ny, nz = wl.grid
    Msize = (2 * nx, 2 * ny, 2 * nz)
    rng = np.random.default_rng(0)
    Gh = (rng.standard_normal((6, Msize[2], Msize[1], Msize[0]))
          + 1j * rng.standard_normal((6, Msize[2], Msize[1], Msize[0])))
    M = np.full((nz, ny, nx), 0.5 + 0.1j)
    x = workloads.random_currents(wl.grid, seed=5)
    return lambda: op.matvec(Gh, wl.grid, M, x)


def _oracle_sample(seconds: float):
    """Oracle matvecs for about `seconds` after one untimed application.
    Returns (matvecs/s, runs, cores)."""
    apply = _oracle_setup()
    apply()
    t0 = time.perf_counter()
    runs = 0
    while True:
        apply()
        runs += 1
        el = time.perf_counter() - t0
        if el >= seconds or runs >= 10000:
            break
    return runs / el, runs, os.cpu_count()


def cpu_baseline(seconds: float):
    v, runs, cores = _oracle_sample(seconds)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{runs} complex128 FFT matvecs of the oracle (scipy.fft, workers={cores}) on the full "
                      f"600x23x11 guide, circulant 1200x46x22, synthetic spectrum; ~{seconds:.0f} s"}


def reference_arm(args):
    """The oracle as the baseline arm: one step is one complex128 oracle
    matvec on the full guide.  W' = min(W, 3) untimed steps, then exactly K'
    timed steps, K' = K capped so that the timed steps take about twice
    --cpu-seconds (a step takes ~0.15 s on 16 cores); the line reports K' and
    W' with the requested K and W beside them."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    apply = _oracle_setup()
    W = min(args.warmup, 3)
    t0 = time.perf_counter()
    for _ in range(max(W, 1)):
        apply()
    per = (time.perf_counter() - t0) / max(W, 1)
    K = int(min(args.steps, max(3, 2 * args.cpu_seconds / per)))
    t0 = time.perf_counter()
    for _ in range(K):
        apply()
    el = time.perf_counter() - t0
    v = K / el
    cores = os.cpu_count()
    result = {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "steps_requested": args.steps, "warmup_requested": getattr(args, "warmup_requested", args.warmup),
        "ms_per_step": 1e3 * el / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD.replace("complex64", "complex128 (FP64 oracle)"), "grid": [600, 23, 11],
                   "circulant": [1200, 46, 22]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{K} oracle FFT matvecs on the full guide after {W} untimed "
                                   f"(requested {args.steps} and {getattr(args, 'warmup_requested', args.warmup)}; capped to ~{2 * args.cpu_seconds:.0f} s)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(result), flush=True)


def studies(args):
    """The parameter studies of Sec. 5 (one JSON line each): R(L) on the
    13.5 um strip for d = 0, 1, 2 at R_rt = 1e-25 and 1e-10 (lengths 450 ..
    9000 nm, reference 9450 nm); electric against matched electric and
    magnetic loss on a 3 um strip (d = 1, 2, lengths 900 .. 4500 nm); and the
    transmission of the 100-period Bragg grating at 101 wavelengths in
    [1.52, 1.57] um."""
    from paper_1803_06237_gb300 import build, sweeps, vie
    build.build_library()
    vie.load()
    if args.rl_sweep:
        lengths = [450.0 * i for i in range(1, 21)]
        for r_rt in (1e-25, 1e-10):
            out = sweeps.rl_sweep(lengths, degrees=(0, 1, 2), r_rt=r_rt, ref_nm=9450.0, tol=1e-8)
            print(json.dumps({"study": "absorber_length", **out}), flush=True)
        # electric + matched magnetic loss on a 3 um strip (JM-VIE, plain GMRES)
        short = [900.0 * i for i in range(1, 6)]
        for matched in (False, True):
            out = sweeps.rl_sweep(short, degrees=(1, 2), r_rt=1e-25, ref_nm=9000.0, tol=1e-8, body_nm=3000.0,
                                  matched=matched)
            print(json.dumps({"study": "absorber_length_matching", **out}), flush=True)
    if args.microring_sweep:
        out = sweeps.microring_sweep(count=args.microring_sweep)
        print(json.dumps({"study": "microring_transmission", **out}), flush=True)
    if args.bragg_sweep:
        lams = [1.52 + 0.0005 * i for i in range(101)]
        out = sweeps.bragg_sweep(lams, periods=100, tol=1e-6, batch=8)
        out["band_gap"] = sweeps.band_gap(out["lambdas_um"], out["T_normalised"])
        print(json.dumps({"study": "bragg_transmission", **out}), flush=True)


def train_study(n_pairs: int, epochs: int):
    """The learned preconditioner at the benchmark's training size: at least
    n_pairs pairs from plain solves of seeded random strips and bends
    (160 x 40 x 11, widths 350-550 nm, up to 20 pairs per problem, problems
    added 100 at a time), `epochs` passes of Adam (mini-batches of 16) with
    the tensor-core training kernels, then on held-out problems: the mean
    loss against the identity's, and flexible GMRES(30) to 1e-6 with the
    judged network against plain GMRES(30), on five random guides and on the
    600 x 23 x 11 benchmark guide."""
    import torch

    from paper_1803_06237_gb300 import build, learned, vie, workloads
    build.build_library()
    vie.load()
    t0 = time.perf_counter()
    pairs, solvers, n_problems = [], [], 0
    while len(pairs) < n_pairs:
        more, solver = learned.make_pairs_many(range(10000 + n_problems, 10000 + n_problems + 100))
        pairs += more
        solvers.append(solver)
        n_problems += 100
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    held, held_solver = learned.make_pairs_many(range(90000, 90020))
    net = vie.vie_net_create(seed=1)
    steps = epochs * len(pairs) // 16
    per_epoch = max(1, len(pairs) // 16)
    t2 = time.perf_counter()
    losses = learned.train(net, pairs, steps=steps, lr=1e-3, batch=16)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    out = {"study": "learned_preconditioner_training", "problems": n_problems, "pairs": len(pairs),
           "grid": [160, 40, 11], "epochs": epochs, "adam_steps": steps, "batch": 16,
           "pair_generation_s": t1 - t0, "train_s": t3 - t2,
           "ms_per_sample": (t3 - t2) * 1e3 / (steps * 16),
           "loss_per_epoch": [float(np.mean(losses[i * per_epoch:(i + 1) * per_epoch])) for i in range(epochs)],
           "identity_loss_train": learned.identity_loss(pairs),
           "held_out": {"pairs": len(held), "identity_loss": learned.identity_loss(held),
                        "network_loss": learned.mean_loss(net, held)}}
    del pairs
    solves = []
    for seed in list(range(90000, 90005)) + [None]:
        wl = workloads.waveguide() if seed is None else workloads.random_guide(seed)
        plan, b = learned.setup_problem(wl)
        row = {"problem": "guide_600x23x11" if seed is None else f"random_guide_{seed}"}
        for name, pc in (("plain", False), ("learned", True)):
            vie.vie_set_preconditioner_net(plan, net if pc else None)
            x = torch.zeros_like(b)
            info = vie.vie_solve(plan, b, x, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30, use_preconditioner=pc,
                                 raise_on_not_converged=False)
            row[name] = {"iterations": info["iterations"], "ms": info["time_ms"], "converged": info["converged"],
                         "dropped": bool(info["fallback"])}
        vie.vie_set_preconditioner_net(plan, None)
        plan.close()
        solves.append(row)
    out["solves"] = solves
    print(json.dumps(out), flush=True)


def profile_train(reps: int):
    """`reps` training samples (forward, loss, backward) of a network with
    random parameters on a random 160 x 40 x 11 guide, tensor-core path: a
    short launch sequence for kernel launch lists.  Prints the time per
    sample (CUDA events)."""
    import torch

    from paper_1803_06237_gb300 import build, learned, vie, workloads
    build.build_library()
    vie.load()
    plan, _ = learned.setup_problem(workloads.random_guide(3))
    n3 = 3 * plan.n_vox
    g = torch.Generator(device="cuda").manual_seed(5)
    r = torch.randn(n3, dtype=torch.complex64, device="cuda", generator=g)
    e = torch.randn(n3, dtype=torch.complex64, device="cuda", generator=g)
    net = vie.vie_net_create(seed=1)
    vie.vie_net_accumulate(net, plan, r, e)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        vie.vie_net_accumulate(net, plan, r, e)
    ev1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_train": reps, "ms_per_sample": ev0.elapsed_time(ev1) / max(reps, 1),
                      "status": vie.vie_net_status(net)}))


def profile_solve(iters: int):
    """One mixed-precision solve of the benchmark guide capped at `iters`
    Arnoldi steps (restart 30), run twice: a short, fixed launch sequence for
    kernel launch lists."""
    import torch

    from paper_1803_06237_gb300 import build, learned, vie, workloads
    build.build_library()
    vie.load()
    plan, b = learned.setup_problem(workloads.waveguide())
    for _ in range(2):
        x = torch.zeros_like(b)
        info = vie.vie_solve(plan, b, x, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30, max_iters=iters,
                             raise_on_not_converged=False)
    print(json.dumps({"profile_solve": iters, "iterations": info["iterations"], "time_ms": info["time_ms"],
                      "graph_cycles": info["graph_cycles"], "reorth_steps": info["reorth_steps"]}))


def profile_net(reps: int):
    """`reps` applications of a network with random parameters on the
    benchmark guide: a short, fixed launch sequence for kernel launch lists."""
    from paper_1803_06237_gb300 import build, learned, vie, workloads
    build.build_library()
    vie.load()
    plan, _ = learned.setup_problem(workloads.waveguide())
    out = net_section(plan, (600, 23, 11), reps=reps)
    print(json.dumps({"profile_net": reps, **out}))


def profile_microring(reps: int):
    """The ring resonator's plan and `reps` complex64 operator applications: a
    short launch sequence for kernel launch lists."""
    import torch

    from paper_1803_06237_gb300 import build, vie, workloads
    build.build_library()
    vie.load()
    wl = workloads.microring()
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps)
    x = torch.randn(3 * wl.n_voxels, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(reps):
        vie.vie_matvec(plan, x, y)
    torch.cuda.synchronize()
    print(json.dumps({"profile_microring": reps, "circulant": list(plan.info()["m"])}))
    plan.close()


def profile_jm(reps: int):
    """The JM-VIE operator (matched permeability) on the benchmark guide:
    `reps` complex64 applications, for kernel launch lists."""
    import torch

    from paper_1803_06237_gb300 import build, learned, vie, workloads
    build.build_library()
    vie.load()
    plan, _ = learned.setup_problem(workloads.waveguide())
    vie.vie_set_permeability(plan, None)
    x = torch.randn(6 * plan.n_vox, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(reps):
        vie.vie_jm_matvec(plan, x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        vie.vie_jm_matvec(plan, x, y)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_jm": reps, "ms_per_matvec": e0.elapsed_time(e1) / reps}))


def profile_circulant(reps: int):
    """Block-circulant builds (complex64 factors, then complex-half factors)
    and `reps` applications of each on the benchmark guide: a short, fixed
    launch sequence for kernel launch lists."""
    import torch

    from paper_1803_06237_gb300 import build, learned, vie, workloads
    build.build_library()
    vie.load()
    plan, b = learned.setup_problem(workloads.waveguide())
    v = torch.randn(b.numel(), dtype=torch.complex64, device="cuda")
    z = torch.empty_like(v)
    setup = {}
    for name, flags in (("complex64", vie.VIE_CIRC_DEFAULT), ("complex_half", vie.VIE_CIRC_FP16_FACTORS)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = vie.vie_circulant_create(plan, flags)
        torch.cuda.synchronize()
        setup[name] = (time.perf_counter() - t0) * 1e3
        for _ in range(reps):
            vie.vie_circulant_apply(c, v, z)
        torch.cuda.synchronize()
        c.close()
    print(json.dumps({"profile_circulant": reps, "setup_ms": setup}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--restart-fp64", type=int, default=200)
    ap.add_argument("--restart-mixed", type=int, default=30)
    ap.add_argument("--train-problems", type=int, default=30)
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--profile-circulant", type=int, default=0,
                    help="only build the block-circulant preconditioner and apply it (for kernel launch lists)")
    ap.add_argument("--profile-microring", type=int, default=0,
                    help="only build the ring resonator's plan and apply the operator (for kernel launch lists)")
    ap.add_argument("--profile-jm", type=int, default=0,
                    help="only run JM-VIE operator applications on the guide (for kernel launch lists)")
    ap.add_argument("--profile-train", type=int, default=0,
                    help="only run tensor-core training samples (for kernel launch lists)")
    ap.add_argument("--profile-net", type=int, default=0,
                    help="only run network applications (for kernel launch lists)")
    ap.add_argument("--no-net", action="store_true")
    ap.add_argument("--no-microring", dest="microring", action="store_false",
                    help="skip the 800 x 600 x 11 ring-resonator operator section")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="create the guide's plan without VIE_PLAN_AUTOTUNE (circulant sizes, x-pass shape)")
    ap.add_argument("--no-circulant", dest="circulant", action="store_false",
                    help="skip the block-circulant preconditioner leg of the solve section")
    ap.add_argument("--rl-sweep", action="store_true",
                    help="only run the absorber-length study of Sec. 5.1 (R(L) and slopes) and print it")
    ap.add_argument("--bragg-sweep", action="store_true",
                    help="only run the Bragg-grating transmission spectrum of Sec. 5.2 and print it")
    ap.add_argument("--microring-sweep", type=int, default=0, metavar="WAVELENGTHS",
                    help="only solve the ring resonator at WAVELENGTHS wavelengths in [1.54, 1.56] um in one batch")
    ap.add_argument("--train-study", type=int, default=0, metavar="PAIRS",
                    help="only train the learned preconditioner on at least PAIRS pairs from random guides and "
                         "measure it on held-out problems")
    ap.add_argument("--train-epochs", type=int, default=3)
    ap.add_argument("--profile-solve", type=int, default=0,
                    help="only run a capped mixed solve (for kernel launch lists)")
    args = ap.parse_args()
    if args.rl_sweep or args.bragg_sweep or args.microring_sweep:
        studies(args)
        return
    if args.train_study:
        train_study(args.train_study, args.train_epochs)
        return
    if args.profile_solve:
        profile_solve(args.profile_solve)
        return
    if args.profile_net:
        profile_net(args.profile_net)
        return
    if args.profile_train:
        profile_train(args.profile_train)
        return
    if args.profile_jm:
        profile_jm(args.profile_jm)
        return
    if args.profile_circulant:
        profile_circulant(args.profile_circulant)
        return
    if args.profile_microring:
        profile_microring(args.profile_microring)
        return
    args.warmup_requested = args.warmup
    if args.warmup < 3:                   # at least three warm-up steps are always run
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
