#!/usr/bin/env python
"""Benchmark of the one-obstacle MFS solution operator on one GB300.

A step is one pass of the whole hot path on the smooth-body workload
(r = 1 + 0.2 sum_j a_j cos js, k = 10, N = 180, M = 216, P = 120, q = 400,
16 seeded plane waves): ring-kernel fill of the 61 distinct modal matrices,
blocked Householder QR of each, then for the 16 waves the incident data,
transform to modes, Q^H, triangular solve and inverse transform to point
strengths.

value = FP64-equivalent algorithmic TFLOP/s of the step: per distinct mode
8 M N^2 - 8 N^3 / 3 (complex QR) plus per wave and mode 16 M N - 4 N^2
(Q^H and back substitution), divided by the device time of the step. The
L2 is flushed (a 256 MB write) before every timed step.

`--impl reference` times the FP64 CPU oracle on the same workload instead.
Multi-GPU (torchrun): each rank runs its own copy of the workload (the
operator's (obstacle, mode) tasks are independent); value sums the ranks'
work over the slowest rank's time ("weak" scaling), no collective on the
data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "operator build time (FP64-equiv TFLOP/s), per-wave apply us at 1e-10 rel err"
FP64_DFMA_PEAK_TFLOPS = 1.195   # measured on this machine's GB300 (profiles/peaks_probe_gb300.md)
# DRAM bytes (read + write) of one split-plan fill on the smooth-body workload
# (fill_samples_kernel 3.0 MB + 261.4 MB, fill_gemm_tc_kernel 319.9 MB + 21.1 MB),
# from the ncu capture in profiles/fill_split_smooth_k10_N180_M216_P120.md. The
# FP64 plans' fill_fft_kernel has no capture of its current form (None).
FILL_TRAFFIC_BYTES = {"split": 3003392 + 261359616 + 319930880 + 21131008, "fp64": None}


def workload():
    wl = synth.config_smooth()
    return wl, wl.obstacles[0]


def step_launches(ob, spec, split, slices):
    """Kernels one step launches, as the library schedules them: fill (split
    plans: sample + digit-GEMM kernel per chunk of ring pairs), per panel step
    the panel, next-panel update and trailing update (split: plus the panel's
    reflector digits, at every step when the plan keeps them for the apply),
    R's digits at the end of a split build, incident, and the apply's RHS
    transform, Q^H, back substitution, scatter and point-strength transform."""
    rows, cols = spec.rows, spec.cols
    D = ob.P // 2 + 1
    npanels = (cols + 15) // 16
    n_next = sum(1 for p in range(npanels) if cols - 16 * (p + 1) > 0)
    n_rest = sum(1 for p in range(npanels) if cols - 16 * (p + 2) > 0)
    n = 1 + npanels + n_next + n_rest + 1 + 5
    if split:
        kinds = 4 if ob.bc != synth.BC_NEUMANN else 1
        L = spec.q // 4 + 1 if (spec.q // 2) % 2 == 0 else (spec.q // 2 + 1) // 2
        Lp = (L + 31) // 32 * 32
        per_pair = 2 * 2 * kinds * 8 * Lp * 2
        chunk = max(8, min(ob.M * ob.N, (512 << 20) // per_pair))
        n += 2 * -(-ob.M * ob.N // chunk) - 1
        kp = (rows + 63) // 64 * 64 + 64
        kept = D * npanels * (4 * slices * 16 * kp * 2 + (16 + kp) * 4) <= (4 << 30)
        n += npanels if kept else n_rest
        n += 1 if (cols + 31) // 32 >= 2 else 0
        n += 0 if kept else 1
    return n


def algorithmic_flops(M, N, P, W):
    D = P // 2 + 1
    qr = D * (8.0 * M * N * N - 8.0 * N ** 3 / 3.0)
    apply = W * P * (16.0 * M * N - 4.0 * N * N)
    return qr, apply


# FP64 issue slots (one slot = one DFMA) of the fill kernel's arithmetic, from
# its source: per ring sample rsqrt (8.2 slots, measured) + the ring sin/cos
# of trig.cuh (the 1024-entry table form, 14 operations) + the products around them (11
# for the normal derivative, 6 for the value kernel); per FFT butterfly the
# adds, multiplies and twiddle products of fft.cuh (radix 2: 8, 3: 22, 4: 28,
# 5: 52); the pruned last stage costs 2 (r - 1) per needed mode.
SINCOS_SLOTS = 14.0
SLOTS_PRODUCTS = {"deriv": 8.2 + 11.0, "value": 8.2 + 6.0}
SLOTS_BUTTERFLY = {2: 8, 3: 22, 4: 28, 5: 52}


def fill_fft_plan(q, D):
    """Radices of the fill's FFT (same rule as the library's plan): 4s, 2, 3,
    5, with the largest radix r with q / r >= D moved last and replaced by
    block sums."""
    rad, m = [], q
    for r in (4, 2, 3, 5):
        while m % r == 0:
            rad.append(r)
            m //= r
    last = None
    cands = [i for i, r in enumerate(rad) if q // r >= D]
    if cands and len(rad) > 1:
        i = max(cands, key=lambda i: rad[i])
        last = rad.pop(i)
    return rad, last


def fill_slots(M, N, P, q, bc_kinds, split):
    """FP64 slots per fill: pairs x ((q/2+1) samples + the transform).
    bc_kinds lists the sample kinds per pair ("deriv" or "value"). Native FP64
    plans transform with the pruned FFT; split plans fold the samples (4 adds
    per folded node) and run the transform on tensor cores (no FP64 slots)."""
    D = P // 2 + 1
    h = q // 2
    if split:
        L = h // 2 + 1 if h % 2 == 0 else (h + 1) // 2
        per_kind = 4.0 * L
    else:
        rad, last = fill_fft_plan(q, D)
        per_kind = sum(SLOTS_BUTTERFLY[r] * (q // r) for r in rad)
        per_kind += 2 * (last - 1) * D if last else 0
    per_pair = sum((h + 1) * (SLOTS_PRODUCTS[k] + SINCOS_SLOTS) + per_kind for k in bc_kinds)
    return M * N * per_pair


class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        # the samples go to $AXI_BENCH_OUT (default: the system temp directory)
        out = os.environ.get("AXI_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_oracle_step(ob, dirs):
    import oracle as O
    coll, src, srcx = O.geometry(ob)
    A, fac = O.factor_operator(ob, coll, src, srcx)
    c = O.solve_modes(ob, fac, O.rhs_modes(O.incident_samples(ob, coll, dirs)))
    O.point_strengths(c, ob.P)
    return c


def cpu_baseline_line(ob, dirs, steps=1):
    """Oracle on the host cores: the whole smooth-body workload (all 61 modes, 16 waves)."""
    qr, ap = algorithmic_flops(ob.M, ob.N, ob.P, dirs.shape[0])
    t0 = time.perf_counter()
    for _ in range(steps):
        run_oracle_step(ob, dirs)
    dt = (time.perf_counter() - t0) / steps
    return {"value": (qr + ap) / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle", "seconds_per_step": dt,
            "sample": f"full workload: fill+QR of {ob.P // 2 + 1} modes, apply of "
                      f"{dirs.shape[0]} waves (numpy FP64, BLAS threads = host cores)"}


def slowest_rank_ms(ms, device):
    """Max over ranks of a per-rank step time: the slowest rank bounds the job.
    Identity without an initialised process group of more than one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, flops_per_rank, ms):
    """Whole-job TFLOP/s: every rank's work over the slowest rank's time."""
    return ws * flops_per_rank / (ms * 1e-3) / 1e12


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="split", choices=["split", "fp64"],
                    help="trailing-update / Q^H arithmetic: Ozaki BF16 digits or native FP64")
    ap.add_argument("--slices", type=int, default=7)
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="launch the step's kernels directly instead of replaying CUDA graphs")
    ap.add_argument("--workload", default="smooth", choices=["smooth", "cup", "batched", "cup_near"],
                    help="smooth (default, the headline line); others print their own line")
    args = ap.parse_args()
    if args.workload != "smooth":
        run_extra_workload(args)
        return
    ws, rank, local = dist_env()
    wl, ob = workload()
    W = wl.n_waves
    dirs_np = synth.plane_wave_directions(W, wl.wave_seed)
    qr_fl, ap_fl = algorithmic_flops(ob.M, ob.N, ob.P, W)
    config = {"workload": wl.name, "precision": args.prec, "obstacle": "smooth r=1+0.2*sum a_j cos(js), seed 2",
              "k": ob.k, "M": ob.M, "N": ob.N, "P": ob.P, "q": ob.q, "waves": W,
              "distinct_modes": ob.P // 2 + 1, "l2": "flushed (256 MB write) before each timed step",
              "launch": "CUDA graph replay" if args.graph else "direct launches"}

    if args.impl == "reference":
        if rank != 0:
            return
        for _ in range(args.warmup):
            run_oracle_step(ob, dirs_np)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            run_oracle_step(ob, dirs_np)
        dt = (time.perf_counter() - t0) / args.steps
        v = (qr_fl + ap_fl) / dt / 1e12
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": os.cpu_count(),
                                 "kind": "oracle", "sample": "full workload per step"},
                "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1506_05083_gb300 import axi

    spec = axi.spec_from_obstacle(ob)
    stream = torch.cuda.current_stream()
    prec = axi.PREC_SPLIT_BF16 | (args.slices << 8) if args.prec == "split" else axi.PREC_FP64
    op = axi.Operator([spec], prec=prec)
    dirs = torch.tensor(dirs_np, device=dev)
    coef = torch.empty((W, ob.P, spec.cols), dtype=torch.complex128, device=dev)
    sigma = torch.empty((W, spec.cols, ob.P), dtype=torch.complex128, device=dev)
    scratch = torch.empty(op.apply_scratch_bytes(W), dtype=torch.uint8, device=dev)
    fill_out = torch.empty((ob.P // 2 + 1, spec.cols, spec.rows), dtype=torch.complex128, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        op.refactor()
        f = op.incident(dirs)
        op.apply(f, want_sigma=True, scratch=scratch, coef=coef, sigma=sigma)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if op.status() != 0:
        raise RuntimeError("device status word set during warm-up")

    # The timed step replays two CUDA graphs captured from the same library
    # calls: the build (fill + look-ahead QR, with its side-stream fork/join)
    # and the apply (incident data, transforms, Q^H, back substitution, point
    # strengths). Inputs and scratch are preallocated; nothing is allocated
    # inside the graphs.
    g_build, g_apply = (torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()) if args.graph else (None, None)
    if args.graph:
        with torch.cuda.graph(g_build):
            op.refactor()
        with torch.cuda.graph(g_apply):
            f_g = op.incident(dirs)
            op.apply(f_g, want_sigma=True, scratch=scratch, coef=coef, sigma=sigma)
        for _ in range(2):
            g_build.replay()
            g_apply.replay()
        torch.cuda.synchronize()
        if op.status() != 0:
            raise RuntimeError("device status word set in graph replay")

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            e0, e1, e2 = evs[i]
            e0.record(stream)
            if args.graph:
                g_build.replay()
            else:
                op.refactor()
            e1.record(stream)
            if args.graph:
                g_apply.replay()
            else:
                f = op.incident(dirs)
                op.apply(f, want_sigma=True, scratch=scratch, coef=coef, sigma=sigma)
            e2.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        # dominant-kernel timing: the fill kernel alone, same stream, L2 flushed
        fev = []
        for i in range(5):
            flush.fill_(i)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            op.fill_modes(out=fill_out)
            b.record(stream)
            fev.append((a, b))
        torch.cuda.synchronize()
    step_ms = [e0.elapsed_time(e2) for e0, _, e2 in evs]
    build_ms = [e0.elapsed_time(e1) for e0, e1, _ in evs]
    apply_ms = [e1.elapsed_time(e2) for _, e1, e2 in evs]
    fill_ms = float(np.mean([a.elapsed_time(b) for a, b in fev]))
    ms = slowest_rank_ms(float(np.mean(step_ms)), dev)
    value = job_value(ws, qr_fl + ap_fl, ms)

    # end to end through the public API with host buffers: H2D of the wave
    # directions from pinned memory, build + apply, D2H of the coefficients
    dirs_host = torch.tensor(dirs_np).pin_memory()
    coef_host = torch.empty((W, ob.P, spec.cols), dtype=torch.complex128).pin_memory()
    e2e = []
    for i in range(max(3, min(args.steps, 10))):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dirs.copy_(dirs_host, non_blocking=True)
        step()
        coef_host.copy_(coef, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e.append(a.elapsed_time(b))
    e2e_ms = slowest_rank_ms(float(np.mean(e2e[1:])), dev)
    h2d = dirs_host.numel() * 8
    d2h = coef_host.numel() * 16

    kinds = ["deriv"] if ob.bc == synth.BC_NEUMANN else ["value", "deriv", "value", "deriv"]
    slots = fill_slots(ob.M, ob.N, ob.P, spec.q, kinds, args.prec == "split")
    ach = 2.0 * slots / (fill_ms * 1e-3) / 1e12          # one slot = one FMA = 2 flops
    launches_per_step = step_launches(ob, spec, args.prec == "split", args.slices)
    torch.cuda.synchronize()
    status = op.status()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "precision": (f"split-bf16 {args.slices} digits (QR trailing updates, Q^H, TRSM off-diagonal "
                          "blocks; fill transform 8 digits); "
                          "fill samples, panels, T, TRSM diagonal blocks, transforms FP64") if args.prec == "split"
                         else "native fp64",
            "build_ms": float(np.mean(build_ms)),
            "build_tflops": qr_fl / (np.mean(build_ms) * 1e-3) / 1e12,
            "apply_us_per_wave": float(np.mean(apply_ms)) * 1e3 / W,
            "e2e": {"value": job_value(ws, qr_fl + ap_fl, e2e_ms), "unit": "TFLOP/s",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": {"kernel": ("fill_samples_kernel + fill_gemm_tc_kernel (FP64 samples, "
                                    "tcgen05 transform)") if args.prec == "split"
                                   else "fill_fft_kernel",
                         "bound": "alu", "achieved": ach,
                         "peak": FP64_DFMA_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_DFMA_PEAK_TFLOPS, "traffic": FILL_TRAFFIC_BYTES[args.prec],
                         "work": "FP64 issue slots of the kernel's arithmetic x 2 flops "
                                 f"({slots:.4g} slots per launch)",
                         "peak_source": "FP64 DFMA probe of measured (MEASURED_PEAKS.json has "
                                        "no FP64 entry)",
                         "kernel_ms": fill_ms},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(),
            "device_status": status,
        }
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline_line(ob, dirs_np)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_extra_workload(args):
    """Device-timed lines for the other workloads (one GPU, CUDA events, L2 flushed):
    cup      cup k=25, N=360, M=432, P=180: build + 16-wave apply per step
    batched  64 seeded obstacles in one plan: build of all + 4 waves applied to each
    cup_near cup factors built once; per step a 256-wave apply + the 3x3 near-image sum
    """
    import torch
    from paper_1506_05083_gb300 import axi
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    prec = axi.PREC_SPLIT_BF16 | (args.slices << 8) if args.prec == "split" else axi.PREC_FP64
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    near_slices = 6
    if args.workload == "batched":
        wl = synth.config_batched()
        specs = [axi.spec_from_obstacle(o) for o in wl.obstacles]
        W = wl.n_waves
    else:
        wl = synth.config_cup() if args.workload == "cup" else synth.config_cup_apply()
        specs = [axi.spec_from_obstacle(wl.obstacles[0])]
        W = wl.n_waves
    op = axi.Operator(specs, prec=prec)
    qr_fl = sum((s.P // 2 + 1) * (8.0 * s.rows * s.cols ** 2 - 8.0 * s.cols ** 3 / 3) for s in specs)
    ap_fl = sum(W * s.P * (16.0 * s.rows * s.cols - 4.0 * s.cols ** 2) for s in specs)
    dirs = torch.tensor(synth.plane_wave_directions(W, wl.wave_seed), device=dev)
    bufs = []
    for i, s in enumerate(specs):
        bufs.append((torch.empty((W, s.P, s.cols), dtype=torch.complex128, device=dev),
                     torch.empty((W, s.cols, s.P), dtype=torch.complex128, device=dev),
                     torch.empty(op.apply_scratch_bytes(W, i), dtype=torch.uint8, device=dev)))
    near = args.workload == "cup_near"
    if near:
        s0 = specs[0]
        near_out = torch.empty((W, s0.M * s0.P), dtype=torch.complex128, device=dev)
        near_scr = torch.empty(axi._near_bytes(op, 0, W, wl.lattice, near_slices), dtype=torch.uint8,
                               device=dev)
        near_fl = 8.0 * 8 * s0.M * s0.P * s0.N * s0.P * W

    def build():
        op.refactor()

    def apply():
        for i in range(len(specs)):
            coef, sigma, scr = bufs[i]
            op.apply(op.incident(dirs, obs=i), obs=i, want_sigma=True, scratch=scr, coef=coef,
                     sigma=sigma)
        if near:
            axi.near_image_sum(op, bufs[0][0], wl.lattice, dirs, slices=near_slices, out=near_out,
                               scratch=near_scr)

    for _ in range(args.warmup):
        if not near:
            build()
        apply()
    torch.cuda.synchronize()
    if op.status() != 0:
        raise RuntimeError("device status word set during warm-up")
    stream = torch.cuda.current_stream()
    tb, ta = [], []
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            if not near:
                build()
            e1.record(stream)
            apply()
            e2.record(stream)
            torch.cuda.synchronize()
            tb.append(e0.elapsed_time(e1))
            ta.append(e1.elapsed_time(e2))
    build_ms = float(np.mean(tb))
    apply_ms = float(np.mean(ta))
    ms = build_ms + apply_ms
    flops = (0.0 if near else qr_fl) + ap_fl + (near_fl if near else 0.0)
    line = {"metric": METRIC, "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "precision": args.prec, "obstacles": len(specs),
                       "waves": W, "l2": "flushed (256 MB write) before each timed step",
                       "near_image_digits": near_slices if near else None},
            "build_ms": None if near else build_ms,
            "build_tflops": None if near else qr_fl / (build_ms * 1e-3) / 1e12,
            "apply_ms": apply_ms, "apply_us_per_wave": apply_ms * 1e3 / W,
            "clocks": clk.summary(), "device_status": op.status()}
    if near:
        line["near_image_pairs_per_s"] = 8.0 * s0.M * s0.P * s0.N * s0.P * W / (apply_ms * 1e-3)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
