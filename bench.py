#!/usr/bin/env python
"""Benchmark of the FP64 band Cholesky factor + solve on one GB300.

Workload (the plain FP64 sweep): single SPD band matrices of order
n = 100000 with half-bandwidth k in {50, 100, 200, 500, 1000, 2000}, A = L0 L0^T
with L0 lower banded, off-diagonals U(-1,1)/sqrt(k), diagonal log-uniform in
[1, 1e3], seed 0, one right-hand side b ~ N(0,1).  One step factors and
solves every matrix of the sweep once.  Inputs are synthetic, generated by
bandgen; the band (k+1 x n) is restored from a pristine device copy and L2
is flushed (a 256 MB write) before each factorization.

value  = sum over k of the Eq. (1) flop count F(n,k) / (wall time of one step)
         (the paper's GFLOP/s convention, Sec. 3.2 and Table 1).
e2e    = the same metric when every step also copies A and b from pinned
         host memory and reads x and info back (the public Python API); the
         copies run on a second stream, each matrix's factorization waiting
         for its own copy, so later copies overlap earlier factorizations.
roofline = the factor kernel: achieved n*k^2 flops per second (CUDA events
         around each factor launch) against the FP64 peak.
cpu_baseline = the serial CPU oracle on a leading block of each matrix,
         extrapolated by F(n,k)/F(n',k).

Multi-GPU: replicas only (one independent sweep per rank); value sums the
ranks' flops over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import bandgen  # noqa: E402
from paper_2305_04635_gb300.flops import band_bytes, flops_eq1, flops_nk2  # noqa: E402

METRIC = "banded Cholesky GFLOP/s and % roofline over n,k; batched/adjoint vs plain"
N_ROWS = 100000
KS = [50, 100, 200, 500, 1000, 2000]
# FP64 peak: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 1.25
HBM_FALLBACK_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
PRECISIONS = {"fp64": 0, "split": 3}
# bf16 MACs per FP64 multiply-add in the split updates: the 28 digit pairs (a + b <= 6) of two
# seven-digit operands.
SPLIT_MACS_PER_FMA = 28
# DRAM bytes (read + write) of one factor launch at n = 20000 for each sweep k, from
# an ncu capture of dram__bytes_read.sum + dram__bytes_write.sum of this kernel;
# traffic is proportional to n at fixed k, so it is scaled by n / 20000.
TRAFFIC_N20000 = {50: 8.4e6, 100: 16.9e6, 200: 35.5e6, 500: 105.3e6, 1000: 258.5e6, 2000: 563.1e6}
# The same for the launches with the split tensor-core updates (tile 32).
TRAFFIC_SPLIT_N20000 = {1000: 258.6e6, 2000: 555.7e6}


def traffic_table(split: bool) -> dict:
    return TRAFFIC_SPLIT_N20000 if split else TRAFFIC_N20000


def measured_bf16_tflops() -> tuple[float, str]:
    """Sustained cuBLAS bf16 rate (the split updates run inside a long step), else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1700.0, "fallback"


def host_cpu() -> dict:
    """Model name and logical core count of the host (for the CPU baseline's context)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu model") or low.startswith("hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
            for line in out.splitlines():
                if line.startswith("Model name") or line.startswith("Vendor ID"):
                    model = line.split(":", 1)[1].strip()
                    if line.startswith("Model name"):
                        break
        except Exception:
            pass
    import platform
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def measured_hbm_gbs() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def roofline_ms(n: int, k: int, hbm_gbs: float) -> float:
    t_flop = flops_nk2(n, k) / (FP64_PEAK_TFLOPS * 1e12)
    t_mem = 2 * band_bytes(n, k) / (hbm_gbs * 1e9)
    return 1e3 * max(t_flop, t_mem)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index: int):
        self.proc = None
        self.idx = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(n: int, ks: list[int]):
    data = {}
    for k in ks:
        L0 = bandgen.l0_band(n, k, seed=0, diag="log1e3")
        A = bandgen.band_product(L0, k)
        B = bandgen.rhs(n, 1, seed=0)[:, 0].copy()
        data[k] = (A, B)
    return data


def run_ours(args, rank: int, world: int, dev: int):
    import paper_2305_04635_gb300 as bchol

    torch.cuda.set_device(dev)
    ks = args.ks
    n = args.n
    data = make_inputs(n, ks)
    stream = torch.cuda.current_stream()
    h = bchol.Handle(tile=args.tile)
    h.set_precision(PRECISIONS[args.precision])
    bufs = {}
    for k in ks:
        A, B = data[k]
        pristine = bchol.band_from_numpy(A)
        work = bchol.band_from_numpy(A)
        host_A = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()   # (n, k+1) == band, column-major
        host_b = torch.from_numpy(B).pin_memory()
        host_x = torch.empty(n, dtype=torch.float64).pin_memory()
        host_info = torch.empty(1, dtype=torch.int32).pin_memory()
        b_pr = torch.from_numpy(B).cuda()
        bufs[k] = dict(pristine=pristine, work=work, b_pr=b_pr, b=b_pr.clone(), info=torch.zeros(1, dtype=torch.int32,
                       device="cuda"), host_A=host_A, host_b=host_b, host_x=host_x, host_info=host_info)
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")
    ev = {k: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for k in ks}
    # Which matrices run the split updates (the library's rule for the automatic tile).
    split_k = {k: args.precision == "split" and (args.tile == 32 or (args.tile == 0 and k > 640)) for k in ks}
    fac_ms = {k: [] for k in ks}
    sol_ms = {k: [] for k in ks}

    def step(record: bool):
        for k in ks:
            bb = bufs[k]
            bb["work"].copy_(bb["pristine"])
            bb["b"].copy_(bb["b_pr"])
            flush.fill_(1.0)
            e0, e1, e2 = ev[k]
            e0.record(stream)
            bchol.factor(bb["work"], k, info=bb["info"], handle=h)
            e1.record(stream)
            bchol.solve(bb["work"], k, bb["b"], handle=h)
            e2.record(stream)
        torch.cuda.synchronize()
        if record:
            for k in ks:
                e0, e1, e2 = ev[k]
                fac_ms[k].append(e0.elapsed_time(e1))
                sol_ms[k].append(e1.elapsed_time(e2))

    copy_stream = torch.cuda.Stream()

    def e2e_step():
        # The inputs of all matrices go up on a copy stream at once; each factorization waits
        # only for its own copy (an event), so later copies overlap earlier factorizations.  The
        # previous step ended with a synchronize, so no buffer is still in use.
        ready = {}
        with torch.cuda.stream(copy_stream):
            for k in ks:
                bb = bufs[k]
                bb["work"].T.copy_(bb["host_A"], non_blocking=True)
                bb["b"].copy_(bb["host_b"], non_blocking=True)
                ready[k] = copy_stream.record_event()
        for k in ks:
            bb = bufs[k]
            stream.wait_event(ready[k])
            bchol.factor(bb["work"], k, info=bb["info"], handle=h)
            bchol.solve(bb["work"], k, bb["b"], handle=h)
            bb["host_x"].copy_(bb["b"], non_blocking=True)
            bb["host_info"].copy_(bb["info"], non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
    # correctness gate on the last warm-up results
    for k in ks:
        rc, infos = bchol.get_info(bufs[k]["info"], handle=h)
        if rc != 0 or infos[0] != 0:
            raise RuntimeError(f"factorization failed for k={k}: status {rc}, info {infos}")

    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(True)
    torch.cuda.synchronize()
    barrier(world)
    t1 = time.perf_counter()
    clk = clocks.stop()
    wall = t1 - t0

    # end-to-end through the public API with host buffers
    for _ in range(1):
        e2e_step()
    barrier(world)
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    te1 = time.perf_counter()
    for k in ks:
        if int(bufs[k]["host_info"][0]) != 0:
            raise RuntimeError(f"e2e factorization failed for k={k}")
    wall_e2e = te1 - te0

    # The same factorizations with FP64-FMA updates, for the matrices that ran the split updates
    # (outside the timed regions).
    fma_ms = {}
    if any(split_k.values()):
        h64 = bchol.Handle(tile=args.tile)
        for k in ks:
            if not split_k[k]:
                continue
            bb = bufs[k]
            times = []
            for _ in range(3):
                bb["work"].copy_(bb["pristine"])
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                bchol.factor(bb["work"], k, info=bb["info"], handle=h64)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            fma_ms[k] = statistics.median(times[1:])
        del h64

    walls = gather_max(world, [wall, wall_e2e])
    wall, wall_e2e = walls
    F = sum(flops_eq1(n, k) for k in ks)
    value = job_rate(world, F, args.steps, wall)
    e2e_value = job_rate(world, F, args.steps, wall_e2e)

    hbm, hbm_kind = measured_hbm_gbs()
    bf16, bf16_kind = measured_bf16_tflops()
    per_k = {}
    tot_flop, tot_ms = 0.0, 0.0
    for k in ks:
        fm = statistics.median(fac_ms[k])
        sm = statistics.median(sol_ms[k])
        roof = roofline_ms(n, k, hbm)
        per_k[str(k)] = {"factor_ms": round(fm, 4), "solve_ms": round(sm, 4),
                         "factor_gflops_eq1": round(flops_eq1(n, k) / fm / 1e6, 2),
                         "factor_gflops_nk2": round(flops_nk2(n, k) / fm / 1e6, 2),
                         "frac_fp64_roofline": round(roof / fm, 4),
                         "dram_bytes": (round(traffic_table(split_k[k])[k] * n / 20000)
                                        if k in traffic_table(split_k[k]) else None),
                         "algorithmic_bytes": 16 * (k + 1) * n,
                         "updates": "split" if split_k[k] else "fp64_fma",
                         # the solve reads the band twice: 16 (k+1) n bytes against the measured HBM copy rate
                         "solve_frac_hbm": round(16 * (k + 1) * n / (hbm * 1e9) * 1e3 / sm, 4)}
        if split_k[k]:
            per_k[str(k)]["factor_ms_fp64_fma"] = round(fma_ms[k], 4)
            per_k[str(k)]["split_speedup"] = round(fma_ms[k] / fm, 3)
            # the split updates' own roofline: 28 bf16 MACs per FP64 FMA of n k^2, against sustained bf16
            per_k[str(k)]["split_tensor_frac"] = round(2 * SPLIT_MACS_PER_FMA * flops_nk2(n, k) / 2 / (fm * 1e-3)
                                                       / (bf16 * 1e12), 4)
        tot_flop += flops_nk2(n, k) * len(fac_ms[k])
        tot_ms += sum(fac_ms[k])
    achieved_tflops = tot_flop / (tot_ms * 1e-3) / 1e12
    ms_per_step = 1e3 * wall / args.steps
    launches_per_step = 3 * len(ks)   # factor kernel + inverse-block kernel + solve kernel per matrix
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"plain FP64 sweep: n={n}, k in {ks}, L0 diag log-uniform [1,1e3], 1 RHS, "
                               "factor + solve per matrix", "n": n, "k": ks, "nrhs": 1,
                   "precision": args.precision,
                   "updates": ("k > 640: FP64-accurate split bf16 products on the tensor cores (tile 32); "
                               "k <= 640: FP64 FMA (tile 16)") if args.precision == "split" else "FP64 FMA",
                   "l2": "256 MB flush write before every factorization (inputs for k <= 100 are below L2 size)",
                   "parallelism": f"replicas x{world}"},
        "per_k": per_k,
        "e2e": {"value": round(e2e_value, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": sum(8 * (k + 1) * n + 8 * n for k in ks),
                "d2h_bytes_per_step": sum(8 * n + 4 for k in ks)},
        "roofline": {"bound": "alu", "achieved": round(achieved_tflops, 4), "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": round(achieved_tflops / FP64_PEAK_TFLOPS, 4),
                     "traffic": (round(sum(traffic_table(split_k[k])[k] for k in ks) * n / 20000 / len(ks))
                                 if all(k in traffic_table(split_k[k]) for k in ks) else None),
                     "traffic_note": "DRAM bytes per factor launch, mean over the sweep's launches (ncu capture at "
                                     "n = 20000, scaled by n); per-k figures in per_k",
                     "kernel": "factor_kernel", "flops_per_launch": "n*k^2",
                     "peak_source": "FP64 nominal from unit counts and clock (alu)",
                     "note": ("achieved counts n*k^2 FP64 multiply-adds as 2 flops each; the k > 640 launches run "
                              "them as split bf16 products on the tensor cores, so their share can pass the FP64 "
                              "ceiling; per_k[k].split_tensor_frac is their tensor-core fraction "
                              f"(bf16 sustained {bf16} TFLOP/s, {bf16_kind})") if any(split_k.values()) else None},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    return out, data


def _ev():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _colmajor(B: np.ndarray) -> torch.Tensor:
    """(n, nrhs) float64 device tensor with column-major strides (ldb = n)."""
    return torch.from_numpy(np.ascontiguousarray(B.T)).cuda().T


def next_batched(count: int = 512, reps: int = 3, precision: int = 3) -> dict:
    """512 independent systems, n log-uniform in [1e3, 5e4], k log-uniform in [50, 400], 4 RHS each:
    one graph-captured batched launch (autotuned tile and CTAs per SM) against a loop of the plain
    per-matrix factor + solve on the same stream.  The batched launch runs in `precision` (split:
    the trailing updates as split products on the tensor cores, in strips) and, for comparison,
    with FP64 FMA updates."""
    import paper_2305_04635_gb300 as bchol
    from paper_2305_04635_gb300 import autotune

    t0 = time.perf_counter()
    ns, ks = bandgen.batch_shapes(count, seed=0)
    pr, bpr = [], []
    for m, (n, k) in enumerate(zip(ns, ks)):
        A = bandgen.band_product(bandgen.l0_band(n, k, 0, "log1e3", matrix_id=m), k)
        pr.append(bchol.band_from_numpy(A))
        bpr.append(_colmajor(bandgen.rhs(n, 4, 0, m)))
    gen_s = time.perf_counter() - t0
    work = [p.clone() for p in pr]
    bw = [b.clone() for b in bpr]
    F = sum(flops_eq1(n, k) for n, k in zip(ns, ks))
    nk2 = sum(flops_nk2(n, k) for n, k in zip(ns, ks))

    def restore():
        torch.cuda.synchronize()          # nothing may still be writing the work copies
        for w, p in zip(work, pr):
            w.copy_(p)
        for w, p in zip(bw, bpr):
            w.copy_(p)
        torch.cuda.synchronize()

    stream = torch.cuda.Stream()
    h = bchol.Handle(stream=stream)
    # plain loop: one warm-up pass over the first systems, then one timed pass over all of them
    with torch.cuda.stream(stream):
        for w, k, b in list(zip(work, ks, bw))[:16]:
            bchol.factor(w, k, handle=h)
            bchol.solve(w, k, b, handle=h)
    restore()
    infos = torch.zeros(count, dtype=torch.int32, device="cuda")
    e0, e1 = _ev()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for m, (w, k, b) in enumerate(zip(work, ks, bw)):
            bchol.factor(w, k, info=infos[m:m + 1], handle=h)
            bchol.solve(w, k, b, handle=h)
        e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    if int(infos.abs().sum()) != 0:
        raise RuntimeError("batched leg: a plain factorization failed")
    x_plain = [b.clone() for b in bw]

    def leg(prec):
        t1 = time.perf_counter()
        classes, member = None, None
        if prec == 3:   # split: the update mode per (n, k) class as well
            plan = autotune.tune_batch_classes(pr, ks, bpr, handle=h)
            tile, cps, classes, member = plan["tile"], plan["ctas_per_sm"], plan["classes"], plan["member_precision"]
        else:
            tile, cps = autotune.tune_batch(pr, ks, bpr, handle=h, precision=prec)
        tune_s = time.perf_counter() - t1
        batch = bchol.Batch(work, ks, bw, tile=tile, ctas_per_sm=cps, precision=prec, member_precision=member)
        restore()
        with torch.cuda.stream(stream):
            batch.run(h)                  # workspace set-up outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            batch.run(h)
        times = []
        for _ in range(reps + 1):
            restore()
            e0, e1 = _ev()
            e0.record(stream)
            with torch.cuda.stream(stream):
                graph.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        batched_ms = statistics.median(times[1:])
        if batch.info.cpu().tolist() != [0] * count:
            raise RuntimeError("batched leg: a batched factorization failed")
        diff = max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(bw, x_plain))
        batch.close()
        # the factorizations alone (a batch without right-hand sides), for the factor / solve split
        fbatch = bchol.Batch(work, ks, None, tile=tile, ctas_per_sm=cps, precision=prec, member_precision=member)
        ftimes = []
        for _ in range(reps + 1):
            restore()
            e0, e1 = _ev()
            e0.record(stream)
            with torch.cuda.stream(stream):
                fbatch.run(h)
            e1.record(stream)
            torch.cuda.synchronize()
            ftimes.append(e0.elapsed_time(e1))
        factor_ms = statistics.median(ftimes[1:])
        fbatch.close()
        return {"batched_ms": round(batched_ms, 3), "batched_factor_ms": round(factor_ms, 3),
                "batched_solve_ms": round(batched_ms - factor_ms, 3),
                "factor_frac_fp64_roofline": round(nk2 / (factor_ms * 1e-3) / (FP64_PEAK_TFLOPS * 1e12), 4),
                "tile": tile, "ctas_per_sm": cps, "max_rel_diff_x_vs_plain": diff, "tune_s": round(tune_s, 1),
                **({"class_modes": {c: ("split" if m == 3 else "fp64") for c, m in classes.items()}}
                   if classes else {})}

    main = leg(precision)
    out = {"workload": f"{count} systems, n log-uniform [1e3,5e4], k log-uniform [50,400], 4 RHS, "
                       "L0 diag log-uniform [1,1e3]",
           "precision": "split" if precision == 3 else "fp64",
           "flops_eq1": F, "plain_loop_ms": round(plain_ms, 3), "speedup_vs_plain": round(plain_ms / main["batched_ms"], 3),
           "batched_gflops_eq1": round(F / main["batched_ms"] / 1e6, 2),
           "factorizations_per_s": round(count / main["batched_ms"] * 1e3, 2),
           "plain_factorizations_per_s": round(count / plain_ms * 1e3, 2), "cuda_graph": True,
           "gen_s": round(gen_s, 1)}
    out.update(main)
    if precision != 0:
        out["fp64_updates"] = leg(0)
    return out


def next_mixed(n: int = 200000, k: int = 1000, nrhs: int = 16, tol: float = 1e-10, reps: int = 2) -> dict:
    """n = 2e5, k = 1000, cond(A) ~ 1e6, 16 RHS: the FP32_UPDATE precision mode through
    bchol_factor / bchol_solve (FP32-accumulated trailing updates, FP64 POTRF, FP64 residual
    refinement to tol), against the FP64 factor + solve with FMA updates and with the split
    (tensor-core) updates.  Each leg is timed with CUDA events, factor and solve apart."""
    import paper_2305_04635_gb300 as bchol

    A = bandgen.band_product(bandgen.l0_band(n, k, 0, "log1e3"), k)
    dA = bchol.band_from_numpy(A)
    b0 = _colmajor(bandgen.rhs(n, nrhs, 0))
    del A

    def leg(precision):
        h = bchol.Handle()
        h.set_precision(precision, max_refine=10, tol=tol)
        fac, sol = [], []
        x = None
        for _ in range(reps + 1):
            ab, b = dA.clone(), b0.clone()
            torch.cuda.synchronize()
            e0, e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), \
                torch.cuda.Event(enable_timing=True)
            e0.record()
            info = bchol.factor(ab, k, handle=h)
            e1.record()
            bchol.solve(ab, k, b, handle=h)
            e2.record()
            torch.cuda.synchronize()
            if int(info.item()) != 0:
                raise RuntimeError(f"mixed leg: factorization failed (precision {precision})")
            fac.append(e0.elapsed_time(e1))
            sol.append(e1.elapsed_time(e2))
            x = b
        out = {"factor_ms": round(statistics.median(fac[1:]), 3), "solve_ms": round(statistics.median(sol[1:]), 3)}
        out["total_ms"] = round(out["factor_ms"] + out["solve_ms"], 3)
        return out, x, h

    fma, x_fma, _ = leg(bchol.FP64)
    split, x_split, _ = leg(bchol.FP64_SPLIT)
    mixed, x_mix, hm = leg(bchol.FP32_UPDATE)
    iters, resid, corr = hm.last_refinement()

    def rel(x, y):
        return float((torch.linalg.norm(x - y, dim=0) / torch.linalg.norm(y, dim=0)).max())

    best = min(fma["total_ms"], split["total_ms"])
    return {"workload": f"n={n}, k={k}, L0 diag log-uniform [1,1e3] (cond ~1e6), {nrhs} RHS",
            "mixed": mixed, "fp64_fma": fma, "fp64_split": split,
            "fp64_factor_solve_ms": fma["total_ms"], "mixed_ms": mixed["total_ms"],
            "speedup_vs_fp64": round(fma["total_ms"] / mixed["total_ms"], 3),
            "speedup_vs_best_fp64": round(best / mixed["total_ms"], 3),
            "refine_tol_rel_residual": tol, "iterations": iters, "final_rel_residual": resid,
            "max_rel_diff_x_vs_fp64": rel(x_mix, x_fma), "max_rel_diff_split_vs_fma": rel(x_split, x_fma)}


def next_adjoint(n: int = 20000, k: int = 200, probe_cols: int = 256, reps: int = 3) -> dict:
    """n = 2e4, k = 200, loss = 0.5 ||A^{-1} b||^2 + log det A: forward (factor, solve, log det) and the
    hand-written backward, against forming the band of A^{-1} from solves with unit vectors (timed on
    probe_cols columns, scaled to n)."""
    import paper_2305_04635_gb300 as bchol
    from paper_2305_04635_gb300.autograd import backward, logdet

    A = bandgen.band_product(bandgen.l0_band(n, k, 0, "log1e3", exact=False), k)
    dA = bchol.band_from_numpy(A)
    b0 = torch.from_numpy(bandgen.rhs(n, 1, 0)[:, 0].copy()).cuda()
    h = bchol.Handle()
    fw, bw, alt = [], [], []
    E = torch.zeros(probe_cols, n, dtype=torch.float64, device="cuda").T
    for _ in range(reps + 1):
        L, x = dA.clone(), b0.clone()
        torch.cuda.synchronize()
        e0, e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), \
            torch.cuda.Event(enable_timing=True)
        e0.record()
        bchol.factor(L, k, handle=h)
        bchol.solve(L, k, x, handle=h)
        ld = logdet(L, handle=h)
        e1.record()
        abar, bbar = backward(L, k, x, x.clone(), 1.0, handle=h)
        e2.record()
        torch.cuda.synchronize()
        fw.append(e0.elapsed_time(e1))
        bw.append(e1.elapsed_time(e2))
        E.zero_()
        E[torch.arange(probe_cols, device="cuda") * (n // probe_cols), torch.arange(probe_cols, device="cuda")] = 1.0
        torch.cuda.synchronize()
        e0, e1 = _ev()
        e0.record()
        bchol.solve(L, k, E, handle=h)
        e1.record()
        torch.cuda.synchronize()
        alt.append(e0.elapsed_time(e1))
    if not bool(torch.isfinite(abar).all()) or not bool(torch.isfinite(ld)):
        raise RuntimeError("adjoint leg: non-finite gradient")
    fw_ms, bw_ms = statistics.median(fw[1:]), statistics.median(bw[1:])
    alt_ms = statistics.median(alt[1:]) * n / probe_cols
    # The band of A^{-1} by the Takahashi recurrences: k multiply-adds for each of the ~n k band
    # entries, 2 n k^2 flops (twice the factorization's n k^2).
    selinv_flops = 2.0 * n * k * k
    return {"workload": f"n={n}, k={k}, loss = 0.5||A^-1 b||^2 + log det A, b ~ N(0,1)",
            "forward_ms": round(fw_ms, 3), "backward_ms": round(bw_ms, 3),
            "backward_over_forward": round(bw_ms / fw_ms, 3),
            "backward_gflops": round(selinv_flops / bw_ms / 1e6, 2),
            "backward_frac_fp64_roofline": round(selinv_flops / (bw_ms * 1e-3) / (FP64_PEAK_TFLOPS * 1e12), 4),
            "backward_flops": "2 n k^2 (band of A^-1 by selected inversion)",
            "alt_inverse_columns_by_solves_ms": round(alt_ms, 3),
            "alt_sample": f"{probe_cols} unit-vector solves, scaled by n/{probe_cols}",
            "speedup_vs_alt": round(alt_ms / bw_ms, 2)}


def cpu_baseline(n: int, ks: list[int], data=None, budget_s: float = 20.0) -> dict:
    """The oracle as it stands on a leading block of each matrix (serial, one core)."""
    import oracle

    oracle.build()
    total_f, total_t = 0.0, 0.0
    samples = []
    per_k_budget = budget_s / len(ks)
    for k in ks:
        # n' rows take about per_k_budget seconds at the oracle's ~0.6 GFLOP/s; at least 2k rows
        nprime = int(min(n, max(2 * k, per_k_budget * 0.6e9 / max(1, (k + 1) * (k + 4)))))
        L0 = bandgen.l0_band(nprime, k, seed=0, diag="log1e3")
        A = bandgen.band_product(L0, k)
        B = bandgen.rhs(nprime, 1, seed=0)[:, 0]
        t0 = time.perf_counter()
        L, info = oracle.pbtrf(A, k)
        oracle.pbtrs(L, k, B)
        dt = time.perf_counter() - t0
        scale = flops_eq1(n, k) / flops_eq1(nprime, k)
        total_f += flops_eq1(n, k)
        total_t += dt * scale
        samples.append(f"k={k}: n'={nprime}")
    return {"value": round(total_f / total_t / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": "factor+solve of the leading n' rows of each matrix, time scaled by F(n,k)/F(n',k): "
                      + ", ".join(samples)}


def measure_peaks() -> dict:
    """Delivered rates of the units behind the roofline denominators (bchol_probe_rate)."""
    import ctypes
    import paper_2305_04635_gb300 as bchol

    h = bchol.Handle()
    out = {}
    for kind, name, iters in [(0, "fp64_dfma", 20000), (1, "fp64_dmma", 4000), (2, "fp32_ffma", 500000),
                              (3, "bf16_tcgen05_mma", 500000)]:
        r = ctypes.c_double()
        rc = h._lib.bchol_probe_rate(h.ptr, kind, iters, ctypes.byref(r))
        out[name + "_tflops"] = round(r.value, 2) if rc == 0 else f"error {rc}"
    out["fp64_nominal_tflops"] = FP64_PEAK_TFLOPS
    return out


def barrier(world: int):
    if world > 1:
        torch.distributed.barrier()


def gather_max(world: int, vals: list[float]) -> list[float]:
    """Element-wise maximum of vals over the ranks (the slowest rank's wall times)."""
    if world == 1:
        return vals
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_rate(world: int, flops_per_rank: float, steps: int, wall: float) -> float:
    """Whole-job GFLOP/s of `world` replicas: every rank's flops over the slowest rank's time."""
    return world * flops_per_rank * steps / wall / 1e9


def batched_case(count: int, n_scale: int, nrhs: int, precision: int, n: int = 0, k: int = 0,
                 reps: int = 3) -> dict:
    """A small batched case for profiling: the batch leg's shape draw (count systems, n divided by
    n_scale) or, with n and k given, that one system; nrhs right-hand sides each (0: factor only);
    tile 32, 2 CTAs/SM.  Runs the plan `reps` times and reports each run's CUDA-event time."""
    import paper_2305_04635_gb300 as bchol

    if n > 0:
        ns, ks = [n], [k]
    else:
        ns, ks = bandgen.batch_shapes(count, seed=0)
        ns = [max(1000, v // n_scale) for v in ns]
    bands = [bchol.band_from_numpy(bandgen.band_product(bandgen.l0_band(nn, kk, 0, "log1e3", matrix_id=m), kk))
             for m, (nn, kk) in enumerate(zip(ns, ks))]
    rhs = [_colmajor(bandgen.rhs(nn, nrhs, 0, m)) for m, nn in enumerate(ns)] if nrhs > 0 else None
    b0 = [b.clone() for b in bands]
    r0 = None if rhs is None else [r.clone() for r in rhs]
    batch = bchol.Batch(bands, ks, rhs, tile=32, ctas_per_sm=2, precision=precision)
    h = bchol.Handle()
    times = []
    for _ in range(reps):
        for b, c in zip(bands, b0):
            b.copy_(c)
        if rhs is not None:
            for r, c in zip(rhs, r0):
                r.copy_(c)
        torch.cuda.synchronize()
        e0, e1 = _ev()
        e0.record()
        batch.run(h)
        e1.record()
        torch.cuda.synchronize()
        times.append(round(e0.elapsed_time(e1), 3))
    if batch.info.cpu().tolist() != [0] * len(ns):
        raise RuntimeError("batched case: a factorization failed")
    batch.close()
    return {"case": "batched", "systems": len(ns), "n_scale": n_scale, "nrhs": nrhs, "ms": times}


def adjoint_case(n: int, k: int, reps: int = 3) -> dict:
    """The adjoint for profiling: factor and solve once, then `reps` backward calls (the solve of
    bbar, the selected inversion, the gradient), each timed with CUDA events."""
    import paper_2305_04635_gb300 as bchol
    from paper_2305_04635_gb300.autograd import backward

    A = bandgen.band_product(bandgen.l0_band(n, k, 0, "log1e3", exact=False), k)
    L = bchol.band_from_numpy(A)
    h = bchol.Handle()
    bchol.factor(L, k, handle=h)
    x = torch.from_numpy(bandgen.rhs(n, 1, 0)[:, 0].copy()).cuda()
    bchol.solve(L, k, x, handle=h)
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = _ev()
        e0.record()
        backward(L, k, x, x.clone(), 1.0, handle=h)
        e1.record()
        torch.cuda.synchronize()
        times.append(round(e0.elapsed_time(e1), 3))
    return {"case": "adjoint", "n": n, "k": k, "backward_ms": times}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_ROWS)
    ap.add_argument("--ks", type=lambda s: [int(x) for x in s.split(",")], default=KS)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-next", action="store_true", help="skip the batched, mixed and adjoint legs")
    ap.add_argument("--tile", type=int, default=0, help="tile size (0: automatic)")
    ap.add_argument("--peaks", action="store_true", help="only measure the FP64/FP32/tensor unit rates and exit")
    ap.add_argument("--precision", default="split", choices=sorted(PRECISIONS),
                    help="trailing-update arithmetic: FP64 FMA, or FP64-accurate split products on the tensor cores")
    ap.add_argument("--case", default="", choices=["", "batched", "adjoint"],
                    help="only run a small case for profiling and print its times (batched: --count systems of the "
                         "batch leg's draw with n divided by --n-scale, or one system with --system n,k; adjoint: "
                         "three backward calls at --system n,k, default 20000,200)")
    ap.add_argument("--count", type=int, default=96)
    ap.add_argument("--n-scale", type=int, default=4)
    ap.add_argument("--nrhs", type=int, default=0)
    ap.add_argument("--system", type=lambda s: [int(x) for x in s.split(",")], default=None)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # The reference arm is the CPU oracle itself (the paper ships no runnable code).
        if rank != 0:
            return
        steps_t = []
        base = None
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            base = cpu_baseline(args.n, args.ks, budget_s=max(2.0, args.cpu_budget / max(1, args.steps)))
            if i >= args.warmup:
                steps_t.append(time.perf_counter() - t0)
        out = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "GFLOP/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.median(steps_t), 3),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic",
               "config": {"workload": f"plain FP64 sweep: n={args.n}, k in {args.ks}, L0 diag log-uniform [1,1e3], "
                                      "1 RHS, factor + solve per matrix", "n": args.n, "k": args.ks, "nrhs": 1},
               "cpu_baseline": base,
               "e2e": {"value": base["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if args.case == "adjoint":
        torch.cuda.set_device(local)
        n, k = args.system if args.system else (20000, 200)
        print(json.dumps(adjoint_case(n, k)))
        return
    if args.case == "batched":
        torch.cuda.set_device(local)
        n, k = args.system if args.system else (0, 0)
        print(json.dumps(batched_case(args.count, args.n_scale, args.nrhs, PRECISIONS[args.precision], n, k)))
        return
    if args.peaks:
        torch.cuda.set_device(local)
        clocks = ClockSampler(local)
        clocks.start()
        peaks = measure_peaks()
        peaks["clocks"] = clocks.stop()
        print(json.dumps(peaks))
        return
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    out, data = run_ours(args, rank, world, local)
    if not args.no_next:
        out["next"] = {"batched": next_batched(precision=PRECISIONS[args.precision]), "mixed": next_mixed(),
                       "adjoint": next_adjoint()}
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.n, args.ks, budget_s=args.cpu_budget)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
