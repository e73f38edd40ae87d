#!/usr/bin/env python
"""Benchmark of the fused Maxwell-Liouville-von Neumann step on GB300.

Workload: three-level medium on a periodic ring, 65536 cells, every cell
active, FP64 (the plain FP64 form); one benchmark step = `--seg` time steps
(default 1000) of the whole grid, so the default 100 steps cover the
workload's 100000 time steps. Metric: cell-updates/s = cells x time steps /
device time (all grid cells, as in the paper's P = N_x N_t / t_exec).

Between timed steps L2 is flushed by writing a 256 MiB buffer (outside the
timed events); the state itself (5.2 MB) would otherwise stay in L2.

--impl reference times the FP64 CPU oracle on bounded samples of the same
workload (it is the only other program here that computes the method).

Multi-GPU: the ring does not shard without a halo exchange, which this
solver does not have; N > 1 runs N independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "cell-updates/sec on 1 GB300 (FP32/batched vs plain FP64 at stated err); % roofline"
UNIT = "cell-updates/s"
WORKLOADS = {
    "three_level_ring": "three-level QCL-like medium, periodic ring, 65536 cells x 100000 steps",
    "six_level_pulse": "six-level manifold (D = 35), Gaussian pulse, hard source + Mur, 1048576 cells x 10000 steps",
    "two_level_sit": "two-level SIT, sech pulse of area 2 pi, 2000 cells x 20000 steps",
    "three_level_ring_pstd": "three-level QCL-like medium, periodic ring, 65536 cells x 100000 steps, "
                             "pseudo-spectral (FFT) field solver",
    "batched": "256 independent devices, N in {2,3,4}, 1k-64k cells (log-uniform), 20000 steps, one graph per call",
    "adjoint": "gradient of the probe energy: three-level ring, 8192 cells x 5000 steps, soft source (512 samples), "
               "checkpoints every 256 steps",
}
WORKLOAD = WORKLOADS["three_level_ring"]


# FP64 and FP32 pipe peaks from unit counts and the maximum SM clock (GB300:
# 152 SMs, 2070 MHz; FP64 1.25 TFLOP/s nominal = 2 DFMA/clk/SM; FP32 128 FFMA/clk/SM).
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_FLOP_PER_CLK_SM = 4
FP32_FLOP_PER_CLK_SM = 256


# DRAM bytes (read + write) per launch of the step kernel from one ncu capture
# (profiles/*.md), keyed by (cell model, precision, workload, steps per launch).
# An entry is used only while the kernel sources hash to the value recorded
# with it; after any change to them the traffic is reported as null.
# dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu, the launch
# shape given), profiles/mln_jit_step_fp64_three_level_ring.md (the default
# run-time compiled kernel) and profiles/mln_jit_step_df32_three_level_ring.md
# (its double-float variant)
MEASURED_TRAFFIC = {
    ("jit", "fp64", "three_level_ring", 8): (5274112.0, "ncu, --block-steps 8 --tile 432"),
    ("jit", "fp64", "three_level_ring", 12): (5273856.0, "ncu, --block-steps 12 --tile 432"),
    ("jit", "fp64", "three_level_ring", 16): (5274112.0, "ncu, --block-steps 16 --tile 432"),
    ("jit", "fp64", "three_level_ring", 20): (5274112.0, "ncu, --block-steps 20 --tile 432"),
    ("df32", "fp64", "three_level_ring", 10): (5295104.0, "ncu, --kernel df32 --block-steps 10 --tile 108"),
}
# sha256 of the sources the measured kernels (the FP64 and double-float step kernels) are
# compiled or generated from, when the counters were taken: a later change of
# one of them makes the reported traffic null until it is measured again
TRAFFIC_SOURCES_SHA = "cc4604d1b315af890cb7c825dacbd0dd290dc4616ea0bded53b9c7668fb6e832"


def kernel_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cuh", "dispatch.cuh", "kernels_fp64.cu", "jit.cu"):
        h.update(open(os.path.join(ROOT, "paper_1710_09799_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic(kernel: str, precision: str, workload: str, block_steps: int):
    if TRAFFIC_SOURCES_SHA is None or kernel_sources_sha() != TRAFFIC_SOURCES_SHA:
        return None
    hit = MEASURED_TRAFFIC.get((kernel, precision, workload, block_steps))
    return None if hit is None else hit[0]


def alu_peak_tflops(precision: str, mhz: float = SM_MAX_MHZ) -> float:
    per = FP64_FLOP_PER_CLK_SM if precision == "fp64" else FP32_FLOP_PER_CLK_SM
    return SMS * per * mhz * 1e6 / 1e12


def pstd_flops_per_step(n: int) -> float:
    """Field part of a PSTD step: two derivatives, each a forward and an inverse
    complex FFT of n points (5 n log2 n flops each, the usual count), the
    spectral multiply (6 n) and the update of the real part (H: n, E: 4 n)."""
    import math
    return 2 * (2 * 5 * n * math.log2(n) + 6 * n) + 5 * n


def pstd_roofline(p, args, run, f_med, clk):
    """Whole-step roofline of the PSTD solver (several kernels per step: the
    medium cell kernel and the FFT passes) against the ALU peak of the
    precision: achieved = (medium flops + FFT flops) per step / step time."""
    steps = args.seg * args.steps
    per_step_s = run["ms"] / 1e3 / steps
    f_step = p.n_medium * f_med + pstd_flops_per_step(p.n_cells)
    achieved = f_step / per_step_s / 1e12
    peak = alu_peak_tflops(args.precision)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "fs_rows_mid + fs_cols + pstd_cell_kernel (whole step)",
            "scope": "whole step: four transform launches and one medium launch per step",
            "flops_per_step": f_step, "fft_flops_per_step": pstd_flops_per_step(p.n_cells),
            "peak_source": f"derived: {SMS} SMs x {FP64_FLOP_PER_CLK_SM if args.precision == 'fp64' else FP32_FLOP_PER_CLK_SM} "
                           f"flop/clk x {SM_MAX_MHZ:.0f} MHz"}


def tensor_roofline(p, args, run, launches, per_launch_s, clk):
    """Roofline of the tensor-core kernel against the TF32 tensor peak (the
    measured sustained bf16 GEMM rate x the nominal TF32 / bf16 ratio 1/2).
    achieved counts the method's two dense products per medium cell update
    (T^T y: 2 D P; [C1, A0^2 T; wm^T, wm^T T] [y; dz]: 2 (D + 1)(D + P)) once;
    issued counts what the MMAs execute (3 x TF32 split, K and N padded to the
    MMA shape, halo rows of every tile)."""
    D, Q = p.D, p.N * (p.N - 1) // 2
    P = 2 * Q
    up = lambda x, m: (x + m - 1) // m * m
    KA, KP, N1, N3 = up(D, 8), up(P, 8), up(P, 16), up(D + 1, 16)
    K, tile = run["shape"][0], run["shape"][1]
    algo_per_cell = 2 * D * P + 2 * (D + 1) * (D + P)
    issued_per_row = 3 * (2 * N1 * KA + 2 * N3 * (KA + KP))
    steps_per_launch = args.seg * args.steps / max(launches, 1)
    ntiles = -(-p.n_cells // tile)
    algo = p.n_medium * algo_per_cell * steps_per_launch / per_launch_s / 1e12
    issued = ntiles * 128 * issued_per_row * steps_per_launch / per_launch_s / 1e12
    peaks = load_peaks()
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    src = "measured bf16_tflops_sustained x 0.5 (nominal tf32 / bf16)"
    if not bf16:
        bf16, src = 1700.0, "fallback 1.7 PFLOP/s bf16 sustained x 0.5"
    peak = 0.5 * bf16
    return {"bound": "tensor", "achieved": algo, "peak": peak, "unit": "TFLOP/s", "frac": algo / peak,
            "kernel": "mln_tc_kernel (tcgen05.mma kind::tf32, 3 x TF32)", "traffic": None, "peak_source": src,
            "issued": issued, "frac_issued": issued / peak, "flops_per_medium_cell_update": algo_per_cell,
            "issued_per_tile_row_step": issued_per_row,
            "counted": "achieved: the two dense products once per medium cell update; issued: MMA work incl. "
                       "split, padding and halo rows"}


def tensor_rotated_roofline(p, args, run, launches, per_launch_s, clk):
    """Roofline of the rotated-basis tensor-core kernel against the FP16 dense
    tensor peak (the measured sustained bf16 GEMM rate: FP16 and bf16 run at
    the same rate). achieved counts the method's one dense product per medium
    cell update, [C1z, cz; wz, cm] [z''; 1]: 2 (D + 1)^2 - (D + 1) flops;
    issued counts what the MMAs execute (hi*hi + hi*lo + lo*hi, K and N padded
    to 16, halo rows of every tile)."""
    D = p.D
    up = lambda x, m: (x + m - 1) // m * m
    KA = NB = up(D + 1, 16)
    K, tile = run["shape"][0], run["shape"][1]
    algo_per_cell = 2 * (D + 1) ** 2 - (D + 1)
    issued_per_row = 3 * 2 * NB * KA
    steps_per_launch = args.seg * args.steps / max(launches, 1)
    ntiles = -(-p.n_cells // tile)
    algo = p.n_medium * algo_per_cell * steps_per_launch / per_launch_s / 1e12
    issued = ntiles * 128 * issued_per_row * steps_per_launch / per_launch_s / 1e12
    peaks = load_peaks()
    fp16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    src = "measured bf16_tflops_sustained (FP16 dense runs at the bf16 rate)"
    if not fp16:
        fp16, src = 1700.0, "fallback 1.7 PFLOP/s bf16 sustained"
    return {"bound": "tensor", "achieved": algo, "peak": fp16, "unit": "TFLOP/s", "frac": algo / fp16,
            "kernel": "mln_tcr_kernel (tcgen05.mma kind::f16, FP16 hi/lo)", "traffic": None, "peak_source": src,
            "issued": issued, "frac_issued": issued / fp16, "flops_per_medium_cell_update": algo_per_cell,
            "issued_per_tile_row_step": issued_per_row,
            "counted": "achieved: the one dense product per medium cell update; issued: MMA work incl. the "
                       "three-part split, padding and halo rows"}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    """The maximum of x over the ranks (CUDA tensor under NCCL, CPU under gloo)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_params(p, precision, form, block_steps=0, tile_cells=0, kernel="auto"):
    from paper_1710_09799_gb300 import mln
    return mln.Params(N=p.N, H0=p.H0, mu=p.mu, G=p.G, rho0=p.rho0, N_a=p.N_a, n_cells=p.n_cells,
                      medium_begin=p.medium_begin, medium_end=p.medium_end, dx=p.dx, dt=p.dt,
                      eps_r=p.eps_r, mu_r=p.mu_r, sigma=p.sigma, boundary=p.boundary,
                      source_kind=p.source_kind, source_cell=p.source_cell, precision=precision, form=form,
                      block_steps=block_steps, tile_cells=tile_cells, kernel=kernel, maxwell=p.maxwell)


def fp32_error_vs_oracle(ref, n_cells=4096, n_steps=2000):
    """The error the FP32 rates come with: E_z (relative, infinity norm) and
    populations (absolute) of the FP32, FP64 and double-float paths (merged
    form) against the FP64 oracle's result `ref` for a 4096-cell ring with the
    parameters of the benchmark ring, after 2000 steps."""
    from paper_1710_09799_gb300 import mln
    q = W.three_level_ring(n_cells=n_cells, n_steps=n_steps)
    out = {"case": f"three-level ring, {n_cells} cells x {n_steps} steps, merged form, against the FP64 oracle"}
    for key, prec, kern in (("fp32", "fp32", "auto"), ("fp64", "fp64", "auto"), ("df32", "fp64", "df32")):
        s = mln.Solver(make_params(q, prec, "merged", kernel=kern), E0=q.e_init())
        s.step(n_steps)
        s.sync()
        E, pops = s.fields()[0], s.populations()
        s.close()
        out[key] = _oracle_error(E, pops, ref)
    return out


def time_device(p, precision, form, seg, steps, warmup, block_steps, tile_cells, ws, flush=True,
                sampler=None, kernel="auto", autotune=True):
    """Device-timed run: returns dict with total ms (max over ranks), launches, shape."""
    import torch
    from paper_1710_09799_gb300 import mln
    s = mln.Solver(make_params(p, precision, form, block_steps, tile_cells, kernel), E0=p.e_init())
    stream = s.stream
    if autotune and not block_steps and not tile_cells:
        s.autotune(3)  # before warm-up, outside the timed region; changes no state
    # source samples of every step of the run, resident on the device
    total = (warmup + steps) * seg
    samples = p.source_samples(0, total)
    src = None if samples is None else torch.as_tensor(samples, dtype=torch.float64, device="cuda")
    seg_src = lambda k: None if src is None else src[k * seg:(k + 1) * seg]
    for w in range(warmup):
        s.step(seg, seg_src(w))
    s.sync()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if flush else None
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = s.launches
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(steps):
            if flush_buf is not None:
                flush_buf.fill_(i & 0xFF)
            evs[i][0].record(stream)
            s.step(seg, seg_src(warmup + i))
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if sampler else None
    barrier(ws)
    s.sync()
    launches = s.launches - l0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms)
    ms_max = max_over_ranks(ws, ms)
    shape = s.launch_shape
    work = s.work_per_step
    kern = s.kernel_in_use
    # d -> rho of every medium cell to host memory (off the stepped path), timed on its own
    rho_ms = None
    if p.n_medium > 0:
        torch.cuda.synchronize()
        t = time.perf_counter()
        s.rho()
        rho_ms = (time.perf_counter() - t) * 1e3
    s.close()
    return dict(ms=ms_max, ms_local=ms, wall_s=t_wall, launches=launches, shape=shape, clocks=clocks, work=work,
                step_ms_median=float(np.median(step_ms)), rho_readout_ms=rho_ms,
                kernel=kern)


def time_batch(precision, seg, steps, warmup, sampler=None, kernel="auto", launch=None):
    """Batched workload: every bench step advances all devices by seg steps (one
    graph launch); launch "chunks" or "persistent" overrides the library's
    default launch structure. Returns the same fields as time_device."""
    import torch
    from paper_1710_09799_gb300 import mln
    total = (warmup + steps) * seg
    devs = W.batched_devices(n_steps=total)
    pars = [make_params(d, precision, "merged", kernel=kernel) for d in devs]
    srcs = [d.source_samples(0, total) for d in devs]
    b = mln.Batch(pars, [d.e_init() for d in devs], srcs, total)
    shape = b.autotune(3)
    if launch is not None:
        b.set_launch(launch)
    for _ in range(warmup):
        b.step(seg)
    b.sync()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stream = b.stream
    l0 = b.shape[3]
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush_buf.fill_(i & 0xFF)
            evs[i][0].record(stream)
            b.step(seg)
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    b.sync()
    ms = sum(a.elapsed_time(c) for a, c in evs)
    launches = b.shape[3] - l0
    cells = sum(d.n_cells for d in devs)
    # algorithmic work per step of every device
    flops = 0.0
    for i, d in enumerate(devs):
        f_med, f_cell, _, _ = mln.mln_work_per_step(mln.mln_batch_context(b.b, i))
        flops += d.n_medium * f_med + d.n_cells * f_cell
    kernels = {N: b.kernel_in_use(N) for N in (2, 3, 4)}
    items = b.shape[2]
    mode = b.launch
    b.close()
    return dict(ms=ms, ms_local=ms, launches=launches, shape=(shape[0], shape[1], items), clocks=clocks,
                cells=cells, flops_per_step=flops, devices=len(devs), kernels=kernels, launch=mode)


def time_e2e(p, precision, form, seg, steps):
    """End to end through the C-ABI with host buffers: each step loads the state
    from pinned host memory, advances seg time steps and reads E_z, H_y back."""
    import torch
    from paper_1710_09799_gb300 import mln
    s = mln.Solver(make_params(p, precision, form), E0=p.e_init())
    s.autotune(3)
    d0, E0, H0 = s.save()
    d_h = torch.from_numpy(d0.reshape(-1).copy()).pin_memory()
    E_h = torch.from_numpy(E0.copy()).pin_memory()
    H_h = torch.from_numpy(H0.copy()).pin_memory()
    E_out = torch.empty_like(E_h).pin_memory()
    H_out = torch.empty_like(H_h).pin_memory()
    dp = lambda t: t.numpy()
    times = []
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        mln.mln_load_state(s.ctx, dp(d_h), dp(E_h), dp(H_h))
        s.step(seg)
        import ctypes as C
        mln._check(mln.lib().mln_get_fields(s.ctx, mln._ptr(dp(E_out)), mln._ptr(dp(H_out))), s.ctx)
        times.append(time.perf_counter() - t)
    s.close()
    t = float(np.sum(times[1:]))
    h2d = d_h.numel() * 8 + E_h.numel() * 8 + H_h.numel() * 8
    d2h = E_out.numel() * 8 + H_out.numel() * 8
    return dict(value=p.n_cells * seg * steps / t, unit=UNIT, h2d_bytes_per_step=h2d,
                d2h_bytes_per_step=d2h, steps=steps, seconds=t)


def cpu_model() -> str:
    """The host CPU's model name (as the kernel reports it), for the baseline record."""
    import platform
    try:
        part = None
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
                if key == "cpu part" and part is None:
                    part = line.split(":", 1)[1].strip()
        if part is not None:  # Arm: the part number (0xd4f: Neoverse V2, as in Grace)
            return f"{platform.machine()} CPU part {part}"
        return platform.processor() or platform.machine()
    except OSError:
        return platform.machine() or "unknown"


def oracle_rate(p, target_s: float, threads: int, max_steps: int = 100000):
    """Oracle cell-updates/s on the full grid for about target_s seconds."""
    import oracle
    oracle.build()
    st = oracle.initial_state(p)
    t = time.perf_counter()
    st, _ = oracle.run(p, st, n_steps=1, threads=threads)
    one = time.perf_counter() - t
    n = int(max(1, min(max_steps, target_s / max(one, 1e-6))))
    t = time.perf_counter()
    oracle.run(p, st, n_steps=n, threads=threads, step0=1)
    dt = time.perf_counter() - t
    return p.n_cells * n / dt, n, dt


def _oracle_error(E, pops, ref, n_cells=None):
    """E_z (relative, infinity norm) and populations (absolute) against an oracle state."""
    E_ref = ref.E if n_cells is None else ref.E[:n_cells]
    p_ref = np.einsum("cii->ci", ref.rho).real
    return {"E_rel": float(np.abs(E - E_ref).max() / max(np.abs(E_ref).max(), 1e-300)),
            "pop_abs": float(np.abs(pops - p_ref[:len(pops)]).max()) if len(pops) else 0.0}


def _fresh_run(p, precision, form, n_steps, kernel="auto"):
    """A fresh solver advanced n_steps from the problem's initial state, in the
    launch shape the autotuner picks (as timed); returns (E, populations)."""
    import torch
    from paper_1710_09799_gb300 import mln
    s = mln.Solver(make_params(p, precision, form, kernel=kernel), E0=p.e_init())
    s.autotune(2)
    smp = p.source_samples(0, n_steps)
    s.step(n_steps, None if smp is None else torch.as_tensor(smp, dtype=torch.float64, device="cuda"))
    s.sync()
    E, _ = s.fields()
    pops = s.populations() if p.n_medium > 0 else np.zeros((0, p.N))
    s.close()
    return E, pops


def _alu_roofline(run, p, seg, steps, precision, kernel_name):
    per_launch_s = run["ms_local"] / 1e3 / max(run["launches"], 1)
    f_med, f_cell, _, _ = run["work"]
    flops = p.n_medium * f_med + p.n_cells * f_cell
    achieved = flops * (seg * steps / max(run["launches"], 1)) / per_launch_s / 1e12
    peak = alu_peak_tflops(precision)
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": None, "kernel": kernel_name, "flops_per_medium_cell_update": f_med,
           "flops_per_grid_cell": f_cell,
           "peak_source": f"derived: {SMS} SMs x {FP64_FLOP_PER_CLK_SM if precision == 'fp64' else FP32_FLOP_PER_CLK_SM} "
                          f"flop/clk x {SM_MAX_MHZ:.0f} MHz"}
    return out


def _kernel_name(kern):
    return "mln_jit_step" if kern == "jit" else ("mln_tc_kernel" if kern == "tensor"
                                                 else f"mln_block_kernel ({kern} cell model)")


def _device_record(p, precision, form, seg, steps, warmup, kernel="auto", note=None, shape=(0, 0)):
    r = time_device(p, precision, form, seg, steps, warmup, shape[0], shape[1], 1, kernel=kernel)
    rec = {"value": p.n_cells * seg * steps / (r["ms"] / 1e3), "unit": UNIT, "ms_per_1000_steps": r["ms"] / (seg * steps) * 1e3,
           "precision": precision, "form": form, "kernel": r["kernel"], "launch_shape": list(r["shape"]),
           "timed": f"{steps} x {seg} time steps after {warmup} x {seg} warm-up, L2 flushed between them"}
    if r["kernel"] == "tensor":
        class _A:  # the arguments the tensor rooflines read
            pass
        a = _A()
        a.seg, a.steps = seg, steps
        per_launch_s = r["ms_local"] / 1e3 / max(r["launches"], 1)
        roof = tensor_rotated_roofline if form == "rotated" else tensor_roofline
        rec["roofline"] = roof(p, a, r, r["launches"], per_launch_s, r["clocks"] or {})
        # the same step's flops (mln_work_per_step) against the FP32 ALU peak, for
        # comparison with the CUDA-core kernels of the same form
        alu = _alu_roofline(r, p, seg, steps, precision, "")
        rec["roofline"]["fp32_alu_equivalent_frac"] = alu["frac"]
    else:
        rec["roofline"] = _alu_roofline(r, p, seg, steps, precision, _kernel_name(r["kernel"]))
    if note:
        rec["roofline"]["note"] = note
    return rec


def oracle_references(threads: int) -> dict:
    """Part of the CPU-baseline leg: the FP64 oracle's results on the host
    cores for the inputs the GPU records below are compared with (each with
    its run time)."""
    import oracle
    oracle.build()
    refs = {}

    def run(key, p, n, **kw):
        t = time.perf_counter()
        refs[key] = oracle.run(p, n_steps=n, threads=threads, **kw) + (time.perf_counter() - t,)

    run("ring_4096", W.three_level_ring(n_cells=4096, n_steps=2000), 2000)
    run("two_level_sit", W.two_level_sit(), 20000)
    run("six_level_4096", W.six_level_pulse(n_cells=4096, n_steps=1000), 1000)
    devs = W.batched_devices(n_steps=1000)
    by_size = sorted(range(len(devs)), key=lambda i: devs[i].n_cells)
    for N in (2, 3, 4):
        i = next(i for i in by_size if devs[i].N == N)
        run(f"batch_device_{i}", devs[i], 1000)
    p = W.adjoint_ring()
    run("adjoint_ring", p, p.n_steps, probe_cell=p.meta["probe_cell"])
    return refs


def workload_records(refs: dict):
    """The other workloads of the benchmark suite, each timed on the device
    (CUDA events, L2 flushed between timed segments) and each with its error
    against the FP64 CPU oracle's results on the same inputs."""
    out = {}
    for section in (_rec_two_level, _rec_six_level, _rec_batched, _rec_adjoint):
        try:
            section(out, refs)
        except Exception as ex:  # keep the benchmark line and the other records
            out[section.__name__[5:]] = {"error": f"{type(ex).__name__}: {ex}"}
    return out


def _rec_two_level(out, refs):
    """two-level SIT (2000 cells x 20000 steps): latency-bound, a parity configuration"""
    p = W.two_level_sit()
    ref, _, t_orc = refs["two_level_sit"]
    for prec in ("fp64", "fp32"):
        rec = _device_record(p, prec, "merged", 2000, 10, 3,
                             note="2000-cell grid: latency-bound; frac_of_one_sm_peak compares with one SM's ALU peak")
        rec["roofline"]["frac_of_one_sm_peak"] = rec["roofline"]["achieved"] / (rec["roofline"]["peak"] / SMS)
        E, pops = _fresh_run(p, prec, "merged", p.n_steps)
        rec["error_vs_oracle"] = dict(_oracle_error(E, pops, ref), case=f"full workload, {p.n_steps} steps",
                                      oracle_s=t_orc)
        out[f"two_level_sit_{prec}"] = rec


def _rec_six_level(out, refs):
    """six-level pulse (1048576 cells): FP32 in its fastest form, FP64 beside it;
    error on a separate 4096-cell x 1000-step run with the same parameters"""
    p = W.six_level_pulse()
    q = W.six_level_pulse(n_cells=4096, n_steps=1000)
    ref, _, t_orc = refs["six_level_4096"]
    # FP64 at a fixed launch shape (autotuning it would take seconds per shape)
    for prec, seg, steps, shape in (("fp32", 500, 5, (0, 0)), ("fp64", 40, 3, (16, 480))):
        rec = _device_record(p, prec, "rotated", seg, steps, 3, shape=shape)
        E, pops = _fresh_run(q, prec, "rotated", q.n_steps)
        rec["error_vs_oracle"] = dict(_oracle_error(E, pops, ref), case="4096 cells x 1000 steps, same parameters",
                                      oracle_s=t_orc)
        out[f"six_level_pulse_{prec}"] = rec


def _rec_batched(out, refs):
    """batched devices (256 grids, N in {2, 3, 4}, 1k-64k cells): the smallest
    grid of each N compared with the oracle after the first 1000 steps; the
    default launch structure (a graph of chunked launches) timed, then the
    persistent launch on the same batch"""
    import torch
    from paper_1710_09799_gb300 import mln
    for prec, seg, steps in (("fp32", 1000, 3), ("fp64", 100, 3)):
        total = 1000 + (4 + 2 * steps) * seg
        devs = W.batched_devices(n_steps=total)
        pars = [make_params(d, prec, "merged") for d in devs]
        srcs = [d.source_samples(0, total) for d in devs]
        b = mln.Batch(pars, [d.e_init() for d in devs], srcs, total)
        b.autotune(2)
        b.step(1000)
        b.sync()
        by_size = sorted(range(len(devs)), key=lambda i: devs[i].n_cells)
        errs = {}
        t_orc = 0.0
        for N in (2, 3, 4):
            i = next(i for i in by_size if devs[i].N == N)
            r, _, t = refs[f"batch_device_{i}"]
            t_orc += t
            E, _ = b.fields(i)
            pops = np.einsum("cii->ci", b.rho(i)).real
            errs[f"device{i}_N{N}_{devs[i].n_cells}_cells"] = _oracle_error(E, pops, r)
        for _ in range(3):
            b.step(seg)
        b.sync()
        flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

        def timed():
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            l0 = b.shape[3]
            torch.cuda.synchronize()
            with torch.cuda.stream(b.stream):
                for i in range(steps):
                    flush_buf.fill_(i & 0xFF)
                    evs[i][0].record(b.stream)
                    b.step(seg)
                    evs[i][1].record(b.stream)
            torch.cuda.synchronize()
            return sum(x.elapsed_time(y) for x, y in evs), b.shape[3] - l0

        ms, launches = timed()
        b.set_launch("persistent")
        b.step(seg)  # capture of the persistent call's graph, outside the timed steps
        b.sync()
        ms_p, launches_p = timed()
        b.sync()
        flops = 0.0
        for i, d in enumerate(devs):
            f_med, f_cell, _, _ = mln.mln_work_per_step(mln.mln_batch_context(b.b, i))
            flops += d.n_medium * f_med + d.n_cells * f_cell
        cells = sum(d.n_cells for d in devs)
        kernels = {N: b.kernel_in_use(N) for N in (2, 3, 4)}
        b.close()
        achieved = flops * seg * steps / (ms / 1e3) / 1e12
        peak = alu_peak_tflops(prec)
        out[f"batched_{prec}"] = {
            "value": cells * seg * steps / (ms / 1e3), "unit": UNIT, "ms_per_1000_steps": ms / (seg * steps) * 1e3,
            "precision": prec, "devices": len(devs), "cells": cells, "cell_model_by_N": kernels,
            "gpu_launches": launches,
            "timed": f"{steps} x {seg} time steps (one graph replay each) after warm-up, L2 flushed between them",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "mln_jit_batch (one launch per N per K steps)"},
            "error_vs_oracle": {"after": "1000 steps", "devices": errs, "oracle_s": t_orc},
            "persistent_launch": {"value": cells * seg * steps / (ms_p / 1e3), "unit": UNIT,
                                  "ms_per_1000_steps": ms_p / (seg * steps) * 1e3, "gpu_launches": launches_p,
                                  "note": "the same batch after mln_batch_set_launch(MLN_BATCH_PERSISTENT): one "
                                          "launch per call and N (mln_jit_batch_persist); not the default"},
        }


def _rec_adjoint(out, refs):
    """gradient workload (8192-cell ring, 5000 steps, checkpoints every 256)"""
    import torch
    from paper_1710_09799_gb300 import mln
    p = W.adjoint_ring()
    src_np = p.source_samples(0, p.n_steps)
    src = torch.as_tensor(src_np, dtype=torch.float64, device="cuda")
    _, probe, t_orc = refs["adjoint_ring"]
    J_orc = p.dt * float(np.sum(probe ** 2))
    rng = np.random.default_rng(0)
    direction = np.zeros(p.n_steps)
    direction[:p.meta["n_src"]] = rng.normal(size=p.meta["n_src"])
    for prec in ("fp64", "fp32"):
        par = make_params(p, prec, "strang")
        times, Js = [], []
        # one context: the initial state reloaded before each evaluation
        # (untimed), the adjoint workspace kept between them
        s = mln.Solver(par, E0=p.e_init())
        s0 = s.save()
        for i in range(3 + 3):
            s.load(*s0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            J, dsrc, dmu, dG = mln.mln_adjoint(s.ctx, p.N, p.n_steps, src.data_ptr(), p.meta["probe_cell"], 256)
            torch.cuda.synchronize()
            if i >= 3:
                times.append(time.perf_counter() - t)
            Js.append(J)
        work = s.work_per_step
        s.close()
        t_grad = float(np.mean(times))
        # the plain forward of the same problem, same precision and form, for the cost ratio
        fwd = time_device(p, prec, "strang", 1000, 3, 2, 0, 0, 1)
        t_fwd = fwd["ms"] / 3e3 * p.n_steps / 1000
        # central difference of the GPU J along one seeded source direction
        h = 1e-6 * np.abs(src_np).max()
        Jpm = []
        for sgn in (1, -1):
            s = mln.Solver(make_params(p, "fp64", "strang"), E0=p.e_init())
            tt = torch.as_tensor(src_np + sgn * h * direction, dtype=torch.float64, device="cuda")
            Jpm.append(mln.mln_adjoint(s.ctx, p.N, p.n_steps, tt.data_ptr(), p.meta["probe_cell"], 10 ** 6)[0])
            s.close()
        fd = (Jpm[0] - Jpm[1]) / (2 * h)
        ad = float(dsrc @ direction)
        f_fwd = p.n_medium * work[0] + p.n_cells * work[1]
        D, Q = p.D, p.N * (p.N - 1) // 2
        rot = 6 * Q + 10 * (Q - (p.N - 1)) + 8 * (p.N - 1)
        # the method's work: the forward step, and the transposed step with the
        # gradients' outer products (A dnb, T^T on the 2q plane rows, T on the
        # plane columns, A yb: 4 D^2 + 8 D q; Dl and T gradients: 4 D^2 + 8 D q;
        # plane terms and the small vectors), not the recomputation
        f_rev = p.n_medium * (8 * D * D + 16 * D * Q + 3 * D + 14 * Q + rot) + p.n_cells * 12
        flops = (f_fwd + f_rev) * p.n_steps
        peak = alu_peak_tflops(prec)
        out[f"adjoint_{prec}"] = {
            "value": p.n_cells * p.n_steps / t_grad, "unit": UNIT + " (forward cell-updates per second of a J + gradient evaluation)",
            "ms_per_gradient": t_grad * 1e3, "gradient_cost_over_forward": t_grad / t_fwd,
            "forward_cell_updates_per_s": p.n_cells * p.n_steps / t_fwd,
            "timed": "3 evaluations after 3 warm-up on one context (host clock around synchronised calls; the "
                     "initial state reloaded before each, untimed; the adjoint workspace kept between them)",
            "J_same_bits_every_evaluation": all(x == Js[0] for x in Js),
            "roofline": {"bound": "alu", "achieved": flops / t_grad / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / t_grad / 1e12 / peak, "traffic": None,
                         "kernel": "whole gradient: forward pass (recording), mln_adjoint_block",
                         "counted": "the forward step (mln_work_per_step) + the transposed step's products and the "
                                    "gradients' outer products, once per medium cell and step"},
            "error_vs_oracle": {"J_rel": abs(J - J_orc) / abs(J_orc), "oracle_s": t_orc,
                                "directional_derivative_vs_central_difference": abs(ad - fd) / max(abs(fd), 1e-300),
                                "direction": "seeded normal over the 512 free source samples, h = 1e-6 max|src| (FP64 forward)"},
        }


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    p = W.three_level_ring()
    threads = os.cpu_count() or 1
    # size each step so that warm-up + steps stay within about two minutes
    st = oracle.initial_state(p)
    t = time.perf_counter()
    oracle.run(p, st, n_steps=1, threads=threads)
    one = time.perf_counter() - t
    per_step_s = min(2.0, 120.0 / max(1, args.steps + args.warmup))
    seg = int(max(1, per_step_s / max(one, 1e-6)))
    for _ in range(args.warmup):
        st, _ = oracle.run(p, st, n_steps=seg, threads=threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        st, _ = oracle.run(p, st, n_steps=seg, threads=threads)
    el = time.perf_counter() - t
    value = p.n_cells * seg * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "n_cells": p.n_cells, "time_steps_per_step": seg,
                   "levels": p.N, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"full 65536-cell ring, {seg} time steps per step, "
                                   f"{args.steps} steps after {args.warmup} warm-up",
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args, ws, rank, local):
    """Gradient workload: each benchmark step is one full J + gradient evaluation
    (forward with checkpoints, backward with recomputation); the value counts the
    forward cell-updates per second of that evaluation."""
    import torch
    from paper_1710_09799_gb300 import mln
    p = W.adjoint_ring()
    src = torch.as_tensor(p.source_samples(0, p.n_steps), dtype=torch.float64, device="cuda")
    par = make_params(p, args.precision, args.form)
    times, Js = [], []
    # one context, as an optimisation loop uses it: the initial state reloaded
    # before each evaluation (untimed), the adjoint workspace kept between them
    s = mln.Solver(par, E0=p.e_init())
    s0 = s.save()
    for i in range(args.warmup + args.steps):
        s.load(*s0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        J, dsrc, dmu, dG = mln.mln_adjoint(s.ctx, p.N, p.n_steps, src.data_ptr(), p.meta["probe_cell"], 256)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
        Js.append(J)
    s.close()
    # the plain forward of the same workload (same form and cell model), for comparison
    s = mln.Solver(par, E0=p.e_init())
    s.autotune(3)
    torch.cuda.synchronize()
    t = time.perf_counter()
    s.step(p.n_steps, src)
    s.sync()
    t_fwd = time.perf_counter() - t
    s.close()
    tot = float(np.sum(times))
    value = ws * p.n_cells * p.n_steps * len(times) / max_over_ranks(ws, tot)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOADS["adjoint"], "n_cells": p.n_cells, "time_steps": p.n_steps,
                   "checkpoint_every": 256, "gradients": "512 source samples, 9 dipole parameters, 81 x 81 G",
                   "evaluations": "one context; initial state reloaded before each (untimed); the adjoint "
                                  "workspace kept between evaluations",
                   "forward_launch_shape": {"block_steps": par.s.block_steps, "tile_cells": par.s.tile_cells}},
        "forward_only_cell_updates_per_s": p.n_cells * p.n_steps / t_fwd,
        "gradient_cost_over_forward": (tot / len(times)) / t_fwd,
        "J": J, "J_same_bits_every_evaluation": all(x == Js[0] for x in Js), "dJ_dmu12": float(dmu[p.N]),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batched(args, ws, rank, local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].isdigit() else local
    prec = args.precision
    r = time_batch(prec, args.seg, args.steps, args.warmup, ClockSampler(smi_index),
                   kernel=args.kernel if args.kernel in ("register", "jit", "df32") else "auto",
                   launch=None if args.batch_launch == "default" else args.batch_launch)
    total_s = max_over_ranks(ws, r["ms"]) / 1e3
    value = ws * r["cells"] * args.seg * args.steps / total_s
    per_launch_s = r["ms"] / 1e3 / max(r["launches"], 1)
    achieved = r["flops_per_step"] * (args.seg * args.steps / max(r["launches"], 1)) / per_launch_s / 1e12
    peak = alu_peak_tflops(prec)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic (seeded devices)",
        "config": {"workload": WORKLOADS["batched"], "devices": r["devices"], "cells": r["cells"],
                   "time_steps_per_step": args.seg, "block_steps": r["shape"][0], "tile_cells": r["shape"][1],
                   "work_items_per_launch": r["shape"][2], "cell_model_by_N": r["kernels"],
                   "launch": r["launch"],
                   "l2": "flushed between steps (256 MiB write)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "kernel": "mln_jit_batch" if "jit" in r["kernels"].values() else "mln_batch_kernel"},
        "gpu_launches": r["launches"], "clocks": r["clocks"],
    }
    if "df32" in r["kernels"].values():
        # double-float pairs run on the FP32 pipe (as the single-grid line)
        p32 = alu_peak_tflops("fp32")
        line["roofline"].update({"kernel": "mln_jit_batch (double-float pairs)", "peak": p32,
                                 "frac": achieved / p32, "frac_of_fp64_peak": achieved / peak})
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="default: fp32 for six_level_pulse and batched, fp64 otherwise")
    ap.add_argument("--form", default=None, choices=["strang", "merged", "rodrigues", "rotated"],
                    help="default: rotated for six_level_pulse (its fastest form), strang for adjoint (the "
                         "form the gradient differentiates), merged otherwise")
    ap.add_argument("--seg", type=int, default=1000, help="time steps per benchmark step")
    ap.add_argument("--block-steps", type=int, default=0, help="0: autotuned")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--kernel", default="auto", choices=["auto", "register", "sparse", "jit", "tensor", "df32"])
    ap.add_argument("--workload", default="three_level_ring", choices=sorted(WORKLOADS))
    ap.add_argument("--quick", action="store_true", help="skip variants, e2e and the CPU baseline")
    ap.add_argument("--batch-launch", default="default", choices=["default", "chunks", "persistent"],
                    help="batched workload: the launch structure (default: the library's)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp32" if args.workload in ("six_level_pulse", "batched") else "fp64"
    if args.form is None:
        args.form = {"six_level_pulse": "rotated", "adjoint": "strang"}.get(args.workload, "merged")
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    from paper_1710_09799_gb300 import build, mln
    if rank == 0 or ws > 1:
        build()
    if args.workload == "batched":
        return run_batched(args, ws, rank, local)
    if args.workload == "adjoint":
        return run_adjoint(args, ws, rank, local)
    p = W.config(args.workload)
    D, q = p.D, p.N * (p.N - 1) // 2

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].isdigit() else local
    sampler = ClockSampler(smi_index)
    main_run = time_device(p, args.precision, args.form, args.seg, args.steps, args.warmup, args.block_steps,
                           args.tile, ws, sampler=sampler, kernel=args.kernel)
    total_s = main_run["ms"] / 1e3
    cell_updates = p.n_cells * args.seg * args.steps
    value = ws * cell_updates / total_s

    # roofline of the fused step kernel (the only kernel in the timed region)
    launches = main_run["launches"]
    per_launch_s = main_run["ms_local"] / 1e3 / max(launches, 1)
    f_med, f_cell, _, _ = main_run["work"]
    flops_per_step = p.n_medium * f_med + p.n_cells * f_cell
    achieved = flops_per_step * (args.seg * args.steps / max(launches, 1)) / per_launch_s / 1e12
    peak = alu_peak_tflops(args.precision)
    kname = ("mln_jit_step" if main_run["kernel"] == "jit" else
             "mln_jit_step (double-float pairs)" if main_run["kernel"] == "df32" else
             f"mln_block_kernel ({main_run['kernel']} cell model)")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "kernel": kname,
                "frac": achieved / peak,
                "traffic": measured_traffic(main_run["kernel"], args.precision, args.workload, main_run["shape"][0]),
                "peak_source": f"derived: {SMS} SMs x {FP64_FLOP_PER_CLK_SM if args.precision == 'fp64' else FP32_FLOP_PER_CLK_SM} "
                               f"flop/clk x {SM_MAX_MHZ:.0f} MHz",
                "flops_per_medium_cell_update": f_med, "flops_per_grid_cell": f_cell,
                "counted": "non-zero entries of the set-up matrices only (mln_work_per_step)"}
    clk = main_run["clocks"] or {}
    if clk.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / alu_peak_tflops(args.precision, clk["sm_mhz"])
    if main_run["kernel"] == "df32":
        # the pairs run on the FP32 pipe: the method's (FP64-equivalent) flops
        # against the FP32 ALU peak, and their ratio to the FP64 peak beside it
        p32 = alu_peak_tflops("fp32")
        roofline.update({"peak": p32, "frac": achieved / p32, "frac_of_fp64_peak": achieved / peak,
                         "peak_source": f"derived: {SMS} SMs x {FP32_FLOP_PER_CLK_SM} flop/clk x {SM_MAX_MHZ:.0f} MHz "
                                        "(FP32: the double-float pairs run on the FP32 pipe)",
                         "note": "achieved counts the method's flops; a pair operation costs 6 to 12 FP32 "
                                 "instructions (ncu: 1378 FP32 thread instructions per computed cell-step, "
                                 "issue 71 % active, FMA pipe 66 %)"})
        if clk.get("sm_mhz"):
            roofline["frac_at_measured_clock"] = achieved / alu_peak_tflops("fp32", clk["sm_mhz"])
    if main_run["kernel"] == "tensor":
        roof = tensor_rotated_roofline if args.form == "rotated" else tensor_roofline
        roofline = roof(p, args, main_run, launches, per_launch_s, clk)
    if p.maxwell == "pstd":
        roofline = pstd_roofline(p, args, main_run, f_med, clk)
    if args.workload == "two_level_sit":
        # 2000 cells fit the shared memory of one SM: a latency-bound parity
        # configuration, also stated against one SM's ALU peak
        roofline["frac_of_one_sm_peak"] = achieved / (peak / SMS)
        roofline["note"] = ("2000-cell grid, latency-bound; frac_of_one_sm_peak compares with the ALU peak "
                            "of one SM")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_run["ms"] / args.steps, "higher_is_better": True,
        "ms_per_step_median": main_run["step_ms_median"], "rho_readout_ms": main_run["rho_readout_ms"],
        "medium_cell_updates_per_s": value * p.n_medium / p.n_cells,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic (seeded: levels, dipoles, rates, noise E^0)",
        "config": {"workload": WORKLOADS[args.workload], "n_cells": p.n_cells, "levels": p.N,
                   "time_steps_per_step": args.seg, "time_steps_total": args.seg * args.steps,
                   "form": args.form, "precision": args.precision, "kernel": main_run["kernel"],
                   "block_steps": main_run["shape"][0], "tile_cells": main_run["shape"][1],
                   "threads_per_block": main_run["shape"][2],
                   "l2": "flushed between steps (256 MiB write); state 5.2 MB stays on chip within a step",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roofline,
        "gpu_launches": launches,
        "clocks": clk,
    }

    if not args.quick and rank == 0 and args.workload == "three_level_ring":
        variants = {}
        for prec, form, kern in (("fp64", "merged", "register"), ("fp64", "strang", "auto"),
                                 ("fp64", "merged", "df32"), ("fp32", "merged", "auto"), ("fp32", "strang", "auto")):
            if (prec, form, kern) == (args.precision, args.form, args.kernel):
                continue
            r = time_device(p, prec, form, args.seg, 10, 2, args.block_steps, args.tile, 1, kernel=kern)
            variants[f"{prec}_{form}_{kern}_shape"] = r["shape"]
            variants[f"{prec}_{form}_{kern}"] = {"value": p.n_cells * args.seg * 10 / (r["ms"] / 1e3), "unit": UNIT,
                                                 "ms_per_step": r["ms"] / 10}
        line["variants"] = variants
        line["e2e"] = time_e2e(p, args.precision, args.form, args.seg, min(10, args.steps))
        if ws == 1:
            threads = os.cpu_count() or 1
            rate, n, secs = oracle_rate(p, 10.0, threads)
            rate1, n1, secs1 = oracle_rate(p, 3.0, 1)  # one thread: the paper's own protocol
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                    "sample": f"full 65536-cell ring, {n} time steps ({secs:.1f} s), FP64",
                                    "cpu_model": cpu_model(),
                                    "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                                      "sample": f"{n1} time steps ({secs1:.1f} s)"}}
            line["vs_oracle"] = value / rate
            # the rest of the CPU-baseline leg: the oracle's results for the
            # error reports of the FP32 variants and of the other workloads
            refs = oracle_references(threads)
            try:
                line["fp32_error_vs_oracle"] = fp32_error_vs_oracle(refs["ring_4096"][0])
            except Exception as ex:  # an auxiliary report: keep the benchmark line
                line["fp32_error_vs_oracle"] = {"error": f"{type(ex).__name__}: {ex}"}
            line["workloads"] = workload_records(refs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
