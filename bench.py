"""Benchmark of the ESP long-range step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl esp|reference]

One step = the whole long-range step on the membrane-slab workload (210,240 atoms,
120 x 120 x 150 A, grid 128 x 128 x 160, P = 6, Delta = 1e-5, r_c = 9 A): wrap + bin/sort,
spread, forward FFT, fused scaling with the energy and 3x3 virial reduction, inverse FFT
and force gather, with inputs resident in HBM.  Every timed step is bracketed by CUDA
events on the plan's stream; the L2 cache is flushed (a 512 MB write) between timed steps
because the workload's inputs are smaller than L2.  Under torchrun (N > 1) each rank runs
an independent replica of the workload on its own GPU (the step has no exchange to
shard), the timed region is bracketed by barriers and rank 0 reports the maximum time.

--impl reference times the FP64 CPU oracle on the host cores instead (see
``reference_arm``).  Both arms print one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "long-range ESP steps/sec and atoms/s at 200k atoms, 1e-5 pressure rel err"
WORKLOAD = "membrane_slab_210k"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# algorithmic bytes (FP32 path): spread reads (s, q) = 16 B per atom and writes one 4 B
# value per grid point; gather reads 16 B per atom and 4 B per grid point and writes 12 B
# of force per atom; scale reads and writes 8 B per half-spectrum mode.
BYTES_PER_ATOM = {"spread": 16, "gather": 28, "bin": 16, "scatter": 16 + 24}
BYTES_PER_POINT = {"spread": 4, "gather": 4}
# FP32 window polynomial degree of the library (Horner, Sec. 4.3)
WINDOW_DEG_F32 = 13
# GB300 unit counts: 128 FP32 lanes per SM (one FMA = 2 FLOP per lane and clock), one
# shared-memory wavefront (32 lanes of 4 B) per SM and clock, SM clock at most 2070 MHz.
# The SM count is read from the device.
FP32_LANES, SM_MAX_MHZ = 128, 2070.0


def algorithmic_ops(kernel: str, P: int):
    """(FLOP, shared-memory accumulations) per atom of spread / gather (FP32 path).

    spread: 3P window values by Horner (2 FLOP per degree), the P^2 products q w1 w2, and
    P^3 products w0 (q w1 w2) accumulated into the tile (P^3 adds).
    gather: 3P window values and 3P derivatives by Horner (2 FLOP per degree each), then
    the separable contraction of the P^3 potential values: sum_i phi w0'_i and
    sum_i phi w0_i per point (2 P^3 multiply-adds), three multiply-adds per (j, k) pair
    and three products per row j.
    """
    d = WINDOW_DEG_F32
    if kernel == "spread":
        return 3 * P * 2 * d + 2 * P * P + 2 * P ** 3, P ** 3
    if kernel == "gather":
        return 6 * P * 2 * d + 2 * (2 * P ** 3 + 3 * P * P + 3 * P), 0
    return None, None


def sm_count(device=0) -> int:
    import torch

    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["esp", "reference"], default="esp")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(synthetic.WORKLOADS), default=WORKLOAD,
                    help="workload to time (the headline metric is quoted on the default)")
    return ap.parse_args(argv)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(my_seconds: float, world: int, device: str) -> float:
    """The slowest rank's time, on every rank (an all-reduce MAX; one process: itself)."""
    if world == 1:
        return my_seconds
    import torch
    import torch.distributed as dist

    t = torch.tensor([my_seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(per_rank_seconds, per_rank_steps):
    """Whole-job throughput: units all ranks processed over the slowest rank's time."""
    t = max(per_rank_seconds)
    return sum(per_rank_steps) / t, t


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(kernel: str, workload: str = WORKLOAD):
    """dram bytes per launch from the committed ncu summary, if it matches this source."""
    import hashlib

    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    src = os.path.join(ROOT, "paper_2601_00161_gb300", "csrc", "esp_kernels.cu")
    try:
        text = open(path).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != digest:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def accuracy_record(workload: str = WORKLOAD):
    """The workload's measured pressure / force errors (FP64 oracle study, committed)."""
    if workload != WORKLOAD:
        return None
    path = os.path.join(ROOT, "tests", "golden", "membrane_slab_accuracy.json")
    try:
        with open(path) as f:
            e = json.load(f)["workload_vs_reference_a"]
    except (OSError, KeyError, ValueError):
        return None
    return {"pressure_diag_rel_err": e["pressure_diag"], "pressure_frobenius_rel_err": e["pressure_frobenius"],
            "pressure_offdiag_rel_err": e["pressure_offdiag"], "forces_rms_rel_err": e["forces_rms"],
            "source": "tests/golden/membrane_slab_accuracy.json (FP64 oracle vs Delta=1e-11 reference)"}


def single_thread():
    """Limit BLAS / OpenMP pools to one thread (the oracle's own work is single-threaded
    numpy either way); a no-op where threadpoolctl is not installed."""
    try:
        from threadpoolctl import threadpool_limits

        return threadpool_limits(1)
    except ImportError:
        import contextlib

        return contextlib.nullcontext()


def cpu_baseline_oracle(S, c):
    """The FP64 oracle as it stands, one full step of the same workload, 1 host thread."""
    from oracle.esp_grid import esp_grid

    with single_thread():
        t0 = time.perf_counter()
        esp_grid(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, forces=True)
        dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"one full oracle step (spread, FFT, scaling, inverse FFT, gather) of "
                      f"{S.name}, {S.n} atoms, FP64, numpy/pocketfft, 1 thread: {dt:.2f} s"}


def cpu_openmp_baseline(S, c, steps=2):
    """The plain OpenMP FP64 ESP (oracle/esp_omp.c) on all host cores, the full workload."""
    from oracle.esp_omp import esp_omp

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    esp_omp(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, threads=cores)  # warm-up (page-in)
    t0 = time.perf_counter()
    for _ in range(steps):
        esp_omp(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, threads=cores)
    dt = (time.perf_counter() - t0) / steps
    return {"value": round(1.0 / dt, 4), "unit": "steps/s", "cores": cores,
            "kind": "plain OpenMP FP64 ESP (oracle/esp_omp.c: spread with atomics, own mixed-radix FFT)",
            "sample": f"{steps} full steps of {S.name} ({S.n} atoms, energy, virial, forces): {dt:.3f} s each"}


def esp_arm(args):
    import torch

    import paper_2601_00161_gb300 as esp

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    S = synthetic.WORKLOADS[args.workload]()
    c = esp.esp_c_from_tolerance(S.delta)
    fp64 = args.precision == "fp64"
    dt = torch.float64 if fp64 else torch.float32
    # a stream of its own: the library captures the step in a CUDA graph (the legacy
    # default stream cannot be captured)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=args.precision,
                    stream=stream.cuda_stream)
    pos = torch.tensor(S.pos, dtype=dt, device="cuda")
    q = torch.tensor(S.q, dtype=dt, device="cuda")
    F = torch.empty((S.n, 3), dtype=dt, device="cuda")
    acc = torch.zeros(esp.ESP_ACCUM_LEN, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        esp.esp_step(plan.handle, pos, q, F, acc)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    # timed region: K steps, the L2 flushed before each, one CUDA event pair per step
    for i in range(args.steps):
        flush.zero_()
        ev0[i].record(stream)
        step()
        ev1[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    # second timed region of K steps with an event before and after every stage (the
    # library records them as nodes of its graph): per-kernel durations for the roofline
    esp.esp_profile(plan.handle, True)
    for _ in range(2):
        step()
    stage_tot = {k: 0.0 for k in esp.STAGES}
    prof_ms = 0.0
    for i in range(args.steps):
        flush.zero_()
        ev0[i].record(stream)
        step()
        ev1[i].record(stream)
        for k, v in esp.esp_profile_read(plan.handle).items():  # synchronises the stream
            stage_tot[k] += v
        prof_ms += ev0[i].elapsed_time(ev1[i])
    clk = clocks.stop()
    esp.esp_profile(plan.handle, False)
    step_ms_prof = prof_ms / args.steps
    my_seconds = sum(step_ms) / 1e3
    # replicas: every rank ran K steps of its own workload; whole-job throughput is all
    # ranks' steps over the slowest rank's time
    t_max = max_over_ranks(my_seconds, world, "cuda")
    value, _ = aggregate([t_max] * world, [args.steps] * world)
    res = esp.esp_result_from_accum(plan.handle, acc.cpu().numpy()).as_dict()

    # dominant kernel of ours and its roofline.  Spread and gather do 30-40 FLOP per
    # algorithmic byte (per atom: ~2 kFLOP against 16-28 B plus 4 B per grid point), above
    # the FP32 ridge of ~12 FLOP/B, so the FP32 path reports them against the FP32 FMA
    # ceiling (unit counts x the maximum SM clock); the FP64 path against HBM.
    ours = ["bin", "spread", "fft_fwd", "xfft_scale", "fft_inv", "gather"]
    avg = {k: stage_tot[k] / args.steps for k in esp.STAGES}
    dom = max(ours, key=lambda k: avg[k])
    Mtot = S.grid[0] * S.grid[1] * S.grid[2]
    sms = sm_count(local)
    peak, peak_kind = measured_peaks()

    def hbm_of(kern):
        b = BYTES_PER_ATOM.get(kern, 16) * S.n + BYTES_PER_POINT.get(kern, 0) * Mtot
        return b * (2 if fp64 else 1)

    fp32_peak_tflops = sms * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    flop_dom, _ = algorithmic_ops(dom, S.P)
    if not fp64 and flop_dom:
        ach = flop_dom * S.n / (avg[dom] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": round(ach, 3),
                    "peak": round(fp32_peak_tflops, 2), "unit": "TFLOP/s",
                    "frac": round(ach / fp32_peak_tflops, 4),
                    "traffic": recorded_traffic(dom, args.workload),
                    "peak_kind": (f"derived: {sms} SMs x {FP32_LANES} FP32 lanes x 2 FLOP x "
                                  f"{SM_MAX_MHZ:.0f} MHz (maximum SM clock)"),
                    "algorithmic_flop": flop_dom * S.n, "algorithmic_bytes": hbm_of(dom),
                    "avg_ms": round(avg[dom], 5)}
    else:
        alg = hbm_of(dom)
        achieved = alg / (avg[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": recorded_traffic(dom, args.workload),
                    "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s",
                    "algorithmic_bytes": alg, "avg_ms": round(avg[dom], 5)}
    # spread and gather against every ceiling: HBM (measured copy bandwidth), FP32 FMA and
    # shared-memory accumulation (unit counts at the sampled SM clock), and the transforms
    # against the HBM copy bandwidth
    sm_hz = 1e6 * (clk.get("sm_mhz") or SM_MAX_MHZ)
    other = {}
    for kern in ("spread", "gather"):
        flop, red = algorithmic_ops(kern, S.P)
        t = avg[kern] * 1e-3
        fp32_peak = sms * FP32_LANES * 2 * sm_hz
        gbs = hbm_of(kern) / t / 1e9
        other[kern] = {"ms": round(avg[kern], 5),
                       "fp32_tflops": round(flop * S.n / t / 1e12, 3),
                       "fp32_frac_at_sampled_clock": round(flop * S.n / t / fp32_peak, 4),
                       "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4)}
        if red:
            red_peak = sms * 32 * sm_hz
            other[kern]["smem_red_per_s"] = round(red * S.n / t, 1)
            other[kern]["smem_red_frac"] = round(red * S.n / t / red_peak, 4)
    # plane transforms: the real grid and the spectrum layout k_xfft works on (the box of
    # the sphere with the library's plane kernels, else cuFFT's full half spectrum)
    info = plan.info()
    H = S.grid[0] * int(info["nb1"]) * int(info["nb2"])
    fft_bytes = (4 if not fp64 else 8) * Mtot + (8 if not fp64 else 16) * H
    for kern in ("fft_fwd", "fft_inv"):
        gbs = fft_bytes / (avg[kern] * 1e-3) / 1e9
        other[kern] = {"ms": round(avg[kern], 5), "bytes": fft_bytes,
                       "kernel": "k_fplane / k_iplane" if info["box_mode"] else "cuFFT plane R2C / C2R",
                       "achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4)}

    # end to end through the public C ABI with host buffers (H2D + step + D2H every step)
    npdt = np.float64 if fp64 else np.float32
    pos_h = torch.tensor(S.pos.astype(npdt)).pin_memory().numpy()
    q_h = torch.tensor(S.q.astype(npdt)).pin_memory().numpy()
    F_h = torch.empty((S.n, 3), dtype=dt).pin_memory().numpy()
    for _ in range(3):
        esp.esp_compute_host(plan.handle, pos_h, q_h, F_h)
    # each call timed on the host clock (the call returns with its results on the host),
    # the L2 flushed before it outside the timed interval
    n_e2e = max(10, min(args.steps, 50))
    e2e_tot = 0.0
    for _ in range(n_e2e):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        esp.esp_compute_host(plan.handle, pos_h, q_h, F_h)
        e2e_tot += time.perf_counter() - t0
    e2e_s = e2e_tot / n_e2e
    e2e = {"value": round(world / e2e_s, 2), "unit": "steps/s",
           "h2d_bytes_per_step": int(pos_h.nbytes + q_h.nbytes),
           "d2h_bytes_per_step": int(F_h.nbytes + 8 * esp.ESP_ACCUM_LEN),
           "l2": "flushed before every call (512 MB write, outside the timed call)"}

    fp64_value = None
    if not fp64 and not args.no_fp64_compare:
        p64 = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision="fp64",
                       stream=stream.cuda_stream)
        pos64 = torch.tensor(S.pos, dtype=torch.float64, device="cuda")
        q64 = torch.tensor(S.q, dtype=torch.float64, device="cuda")
        F64 = torch.empty((S.n, 3), dtype=torch.float64, device="cuda")
        for _ in range(3):
            esp.esp_step(p64.handle, pos64, q64, F64, acc)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        n64 = max(5, min(args.steps, 20))
        for _ in range(n64):
            flush.zero_()
            e0.record(stream)
            esp.esp_step(p64.handle, pos64, q64, F64, acc)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        fp64_value = round(1e3 * n64 / tot, 2)
        p64.close()

    # energy and pressure only (no inverse FFT, no gather: Sec. 4.1), on a plan of its own
    pe = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=args.precision,
                  stream=stream.cuda_stream)
    for _ in range(max(3, args.warmup)):
        esp.esp_step(pe.handle, pos, q, None, acc)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        esp.esp_step(pe.handle, pos, q, None, acc)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    pe.close()
    energy_pressure = {"value": round(1e3 * args.steps / tot, 2), "unit": "steps/s",
                       "ms_per_step": round(tot / args.steps, 5),
                       "step": "bin/sort, spread, forward FFT, scaling + energy/virial reduction"}

    # the near part of the split on the same workload (esp_near; not part of the
    # long-range metric): pair sums within r_c, forces added onto the long-range ones
    near_out = torch.empty(7, dtype=torch.float64, device="cuda")
    for _ in range(2):
        esp.esp_near(plan.handle, pos, q, F, 1, near_out)
    tot = 0.0
    n_near = max(3, min(args.steps, 10))
    for _ in range(n_near):
        flush.zero_()
        e0.record(stream)
        esp.esp_near(plan.handle, pos, q, F, 1, near_out)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    near_ms = tot / n_near
    near_part = {"ms": round(near_ms, 4),
                 "step": "near part of the split (esp_near): device cell list, pairs within r_c, "
                         "energy, virial, forces added onto the long-range ones"}

    launches_per_step = int(plan.info()["launches"])  # the library's own kernels per full step
    out = None
    if rank == 0:
        ms = 1e3 * t_max / args.steps
        out = {
            "metric": METRIC, "value": round(value, 2), "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if not fp64 else "f64", "data": "synthetic",
            "atoms_per_s": round(value * S.n, 1),
            "ns_per_day_equiv_2fs": round(value * 0.1728, 2),
            "config": {"workload": S.name, "atoms": S.n,
                       "cell_A": np.round(S.cell, 4).tolist(),
                       "grid": list(S.grid), "P": S.P, "delta": S.delta, "c": round(c, 6),
                       "r_c_A": S.rc, "step": "energy + 3x3 virial + forces",
                       "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "accuracy": accuracy_record(S.name)},
            # stages 2-4 of the profile are unused since the binning writes the atoms
            # straight into their tiles' slots
            "stage_ms": {k: round(v, 5) for k, v in avg.items()
                         if k not in ("scan", "scatter", "zero_grid")},
            "stage_timing": ("second timed region of the same K steps with a CUDA event before and "
                             f"after every stage; its steps took {step_ms_prof:.5f} ms each"),
            "roofline": roofline,
            "other_bounds": other,
            "energy_pressure_only": energy_pressure,
            "near_part": near_part,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "fp64_path_value": fp64_value,
            "energy_recip": res["energy_recip"],
            # the long-range pressure (Fourier part plus background) a barostat's
            # semi-isotropic coupling sees: lateral P_A and normal P_L, e^2/A^4
            "pressure_semi_long_range": dict(zip(("P_A", "P_L"), (float(v) for v in esp.esp_pressure_coupling(
                np.asarray(res["pressure_recip"]).reshape(3, 3) + res["pressure_bg"] * np.eye(3),
                esp.ESP_COUPLE_SEMI)))),
        }
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline_oracle(S, c)
            out["cpu_openmp_baseline"] = cpu_openmp_baseline(S, c)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return out


def reference_arm(args):
    """FP64 CPU oracle on the host, one thread: each step is one full oracle step of the
    workload (spread, FFT, scaling, inverse FFT, gather of every atom), about 3 s for the
    210,240-atom slab, so W + K steps of a default run finish in minutes."""
    from oracle.esp_grid import esp_grid
    from oracle.pswf import c_from_tolerance

    world, rank, _ = dist_env()
    if rank != 0:
        return None
    S = synthetic.WORKLOADS[args.workload]()
    c = c_from_tolerance(S.delta)
    with single_thread():
        for _ in range(args.warmup):
            esp_grid(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            esp_grid(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc)
        dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = (f"per step one full FP64 oracle step of {S.name} ({S.n} atoms, grid "
              f"{S.grid[0]}x{S.grid[1]}x{S.grid[2]}, P = {S.P}; energy, virial, forces), "
              f"numpy/pocketfft, 1 host thread")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "atoms_per_s": value * S.n,
        "config": {"workload": S.name, "atoms": S.n, "grid": list(S.grid), "P": S.P,
                   "delta": S.delta, "r_c_A": S.rc},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    args = parse_args(argv)
    out = reference_arm(args) if args.impl == "reference" else esp_arm(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
