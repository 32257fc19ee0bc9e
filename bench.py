"""Benchmark: GBS output probabilities per second on one GB300 (or N, weak scaling).

Headline workload: M = 64 modes, Haar-random U (seed 1), r_i ~ U[0.6, 1.0], 4096
collision-free patterns of n = 16 photons, FP64 path, one batched call per step.
`value` = patterns / device time of the step with inputs resident in HBM;
`e2e` = the same through the C ABI with host index lists and host outputs.

Also reported (`extra`): the mixed FP32 path on the same workload, the mixed-n
collision workload (M = 144), the large instances (M = 900, n = 28 and 30) and
the serving loop (Poisson stream, p50/p99 latency), unless --quick.

`--impl reference` times the CPU oracle (plain C, FP64 subset sum with repeated
products, OpenMP over patterns) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

# DRAM bytes (read + write) per launch of haf_subsets_kernel<double> on the
# headline workload, from one ncu capture (profiles/haf_subsets_fp64_m64_n16.md).
# Reported only while the kernel's sources are the ones the capture was taken
# from; any change to them makes the figure stale and the bench reports null.
NCU_TRAFFIC = {"sources_sha256": "b3893c0911fdf91c94646019a9ce2a1895d97f49e64da263ebfd6285d53d6635", "bytes_per_launch": 367626240.0,
               # executed FP64 flops per cycle (DFMA x 2 + DADD + DMUL) over the 608 peak
               "executed_fp64_frac": 0.881}
KERNEL_SOURCES = ("paper_1908_10070_gb300/csrc/haf_subsets.cu", "paper_1908_10070_gb300/csrc/gbs_internal.cuh")


def capture_current():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest() == NCU_TRAFFIC["sources_sha256"]


def measured_traffic():
    return NCU_TRAFFIC["bytes_per_launch"] if capture_current() else None

WORKLOAD = "batched_m64_n16"
WORKLOAD_DESC = "M=64 Haar U seed 1, r~U[0.6,1.0], 4096 collision-free n=16 patterns, "
METRIC = "GBS output probs/sec at n=16/24/30 vs FP64 oracle; p50/p99 request latency"
UNIT = "probs/s"
SMS, SM_MHZ_MAX, FP64_FLOP_PER_CLK_SM = 152, 2070.0, 4.0


def model_flops(n: int) -> float:
    """Algorithmic FP64 flops of one Hafnian: sum_s C(h,s) * 8 (2s)^3 = 64 2^{h-3} h^2 (h+3)."""
    h = n // 2
    if n % 2 or h == 0:
        return 0.0
    return 64.0 * 2.0 ** (h - 3) * h * h * (h + 3)


def fp64_peak_tflops() -> float:
    """FP64 peak from unit counts and clock: 152 SMs x 4 FP64 flop/clk/SM (2 DFMA
    lanes) x 2.07 GHz = 1.26 TFLOP/s (the part's 1.25 TFLOP/s FP64 rating)."""
    return SMS * FP64_FLOP_PER_CLK_SM * SM_MHZ_MAX * 1e6 / 1e12


def chain_sample_flops(n: int, m: int, samples: int) -> float:
    """Algorithmic FP64 flops of `samples` Algorithm 1 samples of n photons over
    m modes, as the library forms them (8 flops per complex multiply-add): per
    step k, the Theorem 1 products Haf(W_sigma) Haf(W_{rho \\ sigma}) over the
    sets rho and sizes |sigma| inside the theorem's ranges (one of each pair
    G(rho, j) = G(rho, |rho| - j); the sets without the new photon once per
    sample on steps of at least 2^24 subsets), the row expansions of the new
    sub-Hafnians of the sizes read (|T'| products each), and the chosen mode's
    cache update (|T'| products for each odd T' of the prefix)."""
    from math import comb

    def in_range(k, mu, ja, jb):
        lo = max(0, 2 * k - n)
        return ja >= lo and jb >= lo and max(0, 3 * k - ja - jb - n) <= mu <= k - max(ja, jb)

    def rho_work(k, c):  # subsets one set rho of size c enumerates
        w = 0
        for ja in range(0, c + 1, 2):
            a, a2 = ja // 2, c // 2 - ja // 2
            used = any(in_range(k, k - c, ja, jb) for jb in range(0, c + 1, 2))
            twin = a2 < a and any(in_range(k, k - c, 2 * a2, jb) for jb in range(0, c + 1, 2))
            if used and not twin:
                w += comb(c, min(ja, c - ja))
        return w

    def count(k, c, part):  # sets of size c: all, with position k-1, without it
        if part == 0:
            return comb(k, c)
        if part == 1:
            return comb(k - 1, c - 1) if c >= 1 else 0
        return comb(k - 1, c)

    macs = 0
    items = samples * m
    for k in range(1, n + 1):
        work = {p: sum(count(k, c, p) * rho_work(k, c) for c in range(0, k + 1, 2)) for p in (0, 1, 2)}
        if items * work[0] >= 1 << 24:
            macs += items * work[1] + samples * work[2]
        else:
            macs += items * work[0]
        sizes = {s for c in range(0, k + 1, 2) for ja in range(0, c + 1, 2) for jb in range(0, c + 1, 2)
                 if in_range(k, k - c, ja, jb) for s in (ja, c - ja)}
        macs += items * sum(comb(k - 1, s - 1) * (s - 1) for s in sizes if s >= 2 and s % 2 == 0)
        if k < n:
            macs += samples * sum(comb(k - 1, t) * t for t in range(1, k, 2))
    return 8.0 * macs


def fp32_peak_tflops() -> float:
    """FP32 peak from unit counts and clock: 152 SMs x 128 FFMA lanes (256 flop)/clk x 2.07 GHz."""
    return SMS * 256.0 * SM_MHZ_MAX * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_patterns(world: int, rank: int):
    """Weak scaling: each rank owns its own 4096 patterns, the rank-th slice of a
    world * 4096 draw from the workload's seeded stream (rank 0 of a one-GPU run
    gets exactly the headline batch). No data moves between ranks."""
    w = W.WORKLOADS[WORKLOAD]
    pats = W.collision_free_patterns(w["m"], w["n"], w["count"] * world, w["seed"] + 100)
    return list(pats[rank * w["count"]:(rank + 1) * w["count"]])


def max_over_ranks(dist, device, *vals):
    """Largest value of each entry over all ranks (the step time of the job)."""
    if dist is None:
        return list(vals)
    import torch

    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def host_cpu() -> str:
    """Architecture, logical cores and CPU model of the host (from /proc/cpuinfo)."""
    import platform

    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and not model:
                    model = ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "%s, %d logical cores, %s" % (platform.machine(), os.cpu_count() or 0, model or "model unknown")


def cpu_baseline(pats, U, r, target_s: float = 12.0):
    """Oracle FP64 subset sum on the host cores over a bounded sample (the
    workload's patterns, repeated in order when the sample exceeds the batch)."""
    import oracle

    B = oracle.build_B(U, r)
    mats = [B[np.ix_(p, p)] for p in pats]
    k = 64
    t0 = time.perf_counter()
    oracle.haf_batch_f64(mats[:k])
    dt = time.perf_counter() - t0
    k2 = int(max(k, k * target_s / max(dt, 1e-6)))
    sample = [mats[i % len(mats)] for i in range(k2)]
    t0 = time.perf_counter()
    oracle.haf_batch_f64(sample)
    dt2 = time.perf_counter() - t0
    cores = oracle.num_threads()
    # one core on the first 64 patterns
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.haf_batch_f64(mats[:k])
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    return {"value": k2 / dt2, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d patterns (the n=16, M=64 batch of %d, cycled), FP64 subset sum, "
                      "OpenMP over patterns, %.1f s" % (k2, len(pats), dt2),
            "single_core_value": k / dt1, "cpu": host_cpu()}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    U, r, pats = W.workload(WORKLOAD)
    import oracle
    oracle.build()
    B = oracle.build_B(U, r)
    mats = [B[np.ix_(p, p)] for p in pats]
    # each step: a bounded sample of the workload, sized so the run stays short
    t0 = time.perf_counter()
    oracle.haf_batch_f64(mats[:8])
    per = (time.perf_counter() - t0) / 8
    k = int(max(8, min(len(mats), 4.0 / max(per, 1e-9) / max(1, args.steps + args.warmup))))
    for _ in range(args.warmup):
        oracle.haf_batch_f64(mats[:k])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.haf_batch_f64(mats[:k])
    dt = time.perf_counter() - t0
    v = k * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC + "FP64", "patterns_per_step": k},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d of %d patterns per step" % (k, len(pats)), "cpu": host_cpu()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="headline workload only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="arithmetic of the headline line (mixed: FP32 terms, compensated sums)")
    ap.add_argument("--profile-workload", default=None,
                    choices=["batched_m64_n16", "mixed_m144", "large_m900", "chain_n16_m256", "chain_n20_m400"],
                    help="no bench line: run that workload's batch --warmup + --steps times in the given "
                         "precision and print its mean time (the command profiler captures run)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_workload:
        return profile_workload(args)

    import torch
    import paper_1908_10070_gb300 as gbs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    U, r, _ = W.workload(WORKLOAD)
    pats = rank_patterns(world, rank)
    K = gbs.build_kernel(torch.from_numpy(U.view(np.float64).copy()).cuda(), torch.from_numpy(r).cuda())
    idx, n, offs = gbs.pack_patterns(pats)
    b = len(pats)
    d_idx = torch.from_numpy(idx).cuda()
    p = torch.zeros(b, dtype=torch.float64, device="cuda")
    lp = torch.zeros_like(p)
    hf = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    er = torch.zeros_like(p)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    prec = gbs.FP64 if args.precision == "fp64" else gbs.MIXED

    def step():
        gbs.prob_batch(K, d_idx, n, offs, prec, stream=stream, p_out=p, logp_out=lp, haf_out=hf, err_out=er)

    # launch shape for n = 16 from the library's autotuner (untimed)
    tuned_rounds = gbs.autotune(16, prec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ks, ke = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ss, se = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for ev in (ks, ke, ss, se):  # torch creates the CUDA event at its first record
        ev.record(stream)
    step_ms, kern_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()  # write 256 MB > L2 between timed steps
            gbs.set_timing_events(ks, ke)
            ss.record(stream)
            step()
            se.record(stream)
            gbs.set_timing_events(None, None)
            se.synchronize()
            step_ms.append(ss.elapsed_time(se))
            kern_ms.append(ks.elapsed_time(ke))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_step = float(np.sum(step_ms)) / args.steps
    t_kern = float(np.mean(kern_ms))
    t_step, t_kern = max_over_ranks(dist, "cuda", t_step, t_kern)
    value = world * b / (t_step * 1e-3)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    hp = np.zeros(b); hl = np.zeros(b); hh = np.zeros(2 * b); he = np.zeros(b)
    for _ in range(2):
        gbs.prob_batch(K, idx, n, offs, prec, p_out=hp, logp_out=hl, haf_out=hh, err_out=he)
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        gbs.prob_batch(K, idx, n, offs, prec, p_out=hp, logp_out=hl, haf_out=hh, err_out=he)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    assert np.array_equal(hh, hf.cpu().numpy()), "host and device paths disagree"

    flops = model_flops(16) * b
    peak = fp64_peak_tflops() if prec == gbs.FP64 else fp32_peak_tflops()
    achieved = flops / (t_kern * 1e-3) / 1e12
    # the FP64 pipe's measured throughput (DFMA microbenchmark in the library),
    # with the clocks it ran at: the second denominator of the fraction
    with ClockSampler(local) as pclk:
        measured_peak = gbs.measure_fp64_peak()
    pclk_s = pclk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == gbs.FP64 else "f32 terms, f32x2/f64 sums",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC + ("FP64" if prec == gbs.FP64 else "mixed precision"),
                   "patterns_per_step": b, "l2": "flushed (256 MB write) between timed steps",
                   "autotuned_rounds_per_item": tuned_rounds},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": measured_traffic() if prec == gbs.FP64 else None,
                     # the same capture's executed FP64 rate (the flop model above counts
                     # one N x N complex product per subset; the route executes more)
                     "ncu_executed_fp64_frac": (NCU_TRAFFIC["executed_fp64_frac"]
                                                if prec == gbs.FP64 and capture_current() else None),
                     "hafnian_terms_per_s": b * (2 ** 8 - 1) / (t_kern * 1e-3),
                     "kernel": "haf_subsets_kernel<%s>" % ("double" if prec == gbs.FP64 else "float"),
                     "kernel_ms": t_kern,
                     "flops_per_launch": flops,
                     "peak_note": ("FP64 from unit counts and clock (152 SM x 4 flop/clk x 2.07 GHz)"
                                   if prec == gbs.FP64 else
                                   "FP32 from unit counts and clock (152 SM x 256 flop/clk x 2.07 GHz)"),
                     "measured_fp64_peak": measured_peak,
                     "frac_of_measured_fp64_peak": (achieved / measured_peak) if prec == gbs.FP64 else None,
                     "measured_peak_note": "gbs_measure_fp64_peak (independent DFMA chains on every SM), "
                                           "SM clock %s MHz during it" % pclk_s.get("sm_mhz")},
        "e2e": {"value": world * b / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(idx.nbytes),
                "d2h_bytes_per_step": int(hp.nbytes + hl.nbytes + hh.nbytes + he.nbytes)},
        # per step: the route choice, pair terms and repeated-row kernel (FP64
        # only), the subset kernel, finalisation
        "gpu_launches": (5 if prec == gbs.FP64 else 2) * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1 and prec == gbs.FP64:
        line["cpu_baseline"] = cpu_baseline(pats, U, r)
    # the other workloads, serving and the samplers: one-GPU runs only (a
    # multi-rank run holds every GPU meanwhile)
    if rank == 0 and not args.quick and world == 1:
        line["extra"] = extras(gbs, torch, measured_peak)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def timed_batch(gbs, torch, K, pats, precision, reps=3, warm=1, nvtx=None):
    idx, n, offs = gbs.pack_patterns(pats)
    b = len(pats)
    d_idx = torch.from_numpy(idx).cuda()
    p = torch.zeros(b, dtype=torch.float64, device="cuda")
    hf = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    er = torch.zeros_like(p)
    ks, ke = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ks.record()
    ke.record()
    for _ in range(warm):
        gbs.prob_batch(K, d_idx, n, offs, precision, p_out=p, haf_out=hf, err_out=er)
    torch.cuda.synchronize()
    ts, tk = [], []
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gbs.set_timing_events(ks, ke)
        s.record()
        gbs.prob_batch(K, d_idx, n, offs, precision, p_out=p, haf_out=hf, err_out=er)
        e.record()
        gbs.set_timing_events(None, None)
        e.synchronize()
        ts.append(s.elapsed_time(e))
        tk.append(ks.elapsed_time(ke))
    if nvtx:
        torch.cuda.nvtx.range_pop()
    h = hf.cpu().numpy()
    return float(np.median(ts)), float(np.median(tk)), h[0::2] + 1j * h[1::2], er.cpu().numpy()


def stored_oracle(name):
    """Stored double-double oracle Hafnians of a workload (tests/golden, written
    by the oracle alone), or None when they come from another Haar draw."""
    import hashlib

    U, _, _ = W.workload(name)
    fname = {"large_m900": "large_m900_oracle.json"}.get(name, name + "_oracle.json")
    try:
        with open(os.path.join(ROOT, "tests", "golden", fname)) as f:
            g = json.load(f)
    except OSError:
        return None
    if g.get("U_sha256") != hashlib.sha256(np.ascontiguousarray(U, dtype=np.complex128).tobytes()).hexdigest():
        return None
    if "patterns" in g:
        return np.array([complex(q["haf_dd"][0] + q["haf_dd"][1], q["haf_dd"][2] + q["haf_dd"][3])
                         for q in g["patterns"]])
    return np.array(g["haf_re"]) + 1j * np.array(g["haf_im"])


def error_columns(ref, h, e, tag):
    """Each result's relative error against the oracle and its stated bound."""
    if ref is None:
        return {tag + "_vs_oracle": "unavailable (stored values from another Haar draw)"}
    err = np.abs(h - ref) / np.abs(ref)
    return {tag + "_max_rel_err_vs_oracle": float(err.max()), tag + "_median_rel_err_vs_oracle": float(np.median(err)),
            tag + "_max_stated_bound": float(e.max()), tag + "_within_bound": bool(np.all(err <= e)),
            tag + "_max_err_over_bound": float(np.max(err / e))}


def oracle_rate(pats, U, r, target_s=6.0):
    """CPU baseline of one workload: the oracle's FP64 subset sum on all host
    cores over a bounded sample (the workload's patterns in order, cycled), and
    on one core over its first patterns."""
    import oracle

    B = oracle.build_B(U, r)
    mats = [B[np.ix_(p, p)] for p in pats]
    k = min(len(mats), max(1, oracle.num_threads()))
    t0 = time.perf_counter()
    oracle.haf_batch_f64(mats[:k])
    dt = time.perf_counter() - t0
    k2 = int(max(k, min(len(mats) * 4, k * target_s / max(dt, 1e-6))))
    sample = [mats[i % len(mats)] for i in range(k2)]
    t0 = time.perf_counter()
    oracle.haf_batch_f64(sample)
    dt2 = time.perf_counter() - t0
    cores = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        k1 = min(len(mats), 4)
        t0 = time.perf_counter()
        oracle.haf_batch_f64(mats[:k1])
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    return {"value": k2 / dt2, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d patterns (the workload's %d, in order, cycled), FP64 subset sum, %.1f s"
                      % (k2, len(pats), dt2),
            "single_core_value": k1 / dt1, "cpu": host_cpu()}


def profile_workload(args):
    """One workload's batch, device inputs, repeated: a small, self-contained
    command for profiler captures (-s skips the warm-up launches)."""
    import torch
    import paper_1908_10070_gb300 as gbs

    if args.profile_workload.startswith("chain_"):
        return profile_chain(args, torch, gbs)
    U, r, pats = W.workload(args.profile_workload)
    prec = gbs.FP64 if args.precision == "fp64" else gbs.MIXED
    K = gbs.build_kernel(U, r)
    # the launch shapes the bench uses; the timed steps run inside the NVTX
    # range "timed" (ncu --nvtx --nvtx-include timed/ captures only those)
    tuned = {"batched_m64_n16": (16,), "mixed_m144": tuple(range(8, 25, 2)), "large_m900": (28, 30)}
    for nn in tuned[args.profile_workload]:
        gbs.autotune(nn, prec)
    t = timed_batch(gbs, torch, K, pats, prec, reps=max(1, args.steps), warm=max(0, args.warmup), nvtx="timed")[0]
    print(json.dumps({"workload": args.profile_workload, "precision": args.precision, "patterns": len(pats),
                      "warmup": args.warmup, "steps": args.steps, "ms_per_batch": t}))


def profile_chain(args, torch, gbs):
    """Algorithm 1 chain samples (n photons, m = n^2 modes, r = 0.8814): the
    warm-up samples, then the timed ones inside the NVTX range "timed"."""
    n = int(args.profile_workload.split("_")[1][1:])
    m = n * n
    K = gbs.build_kernel(W.haar_unitary(m, 40 + n), np.full(m, 0.8814))
    rng = np.random.default_rng(n)
    for _ in range(max(0, args.warmup)):
        gbs.sample_chain(K, n, rng.random(n))
    torch.cuda.synchronize()
    ts = []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        gbs.sample_chain(K, n, rng.random(n))
        ts.append(time.perf_counter() - t0)
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"workload": args.profile_workload, "warmup": args.warmup, "steps": len(ts),
                      "ms_per_sample": 1e3 * float(np.median(ts))}))


def extras(gbs, torch, measured_peak):
    out = {}
    peak = fp64_peak_tflops()

    def frac(fl, ms):
        a = fl / (ms * 1e-3) / 1e12
        return {"achieved_tflops": a, "frac_of_nominal_peak": a / peak,
                "frac_of_measured_peak": (a / measured_peak) if measured_peak else None}

    # mixed path on the headline workload
    U, r, pats = W.workload(WORKLOAD)
    ref = stored_oracle(WORKLOAD)
    K = gbs.build_kernel(U, r)
    gbs.autotune(16, gbs.MIXED)
    t64, k64, h64, e64 = timed_batch(gbs, torch, K, pats, gbs.FP64)
    t32, k32, h32, e32 = timed_batch(gbs, torch, K, pats, gbs.MIXED)
    out["n16_mixed"] = {"probs_per_s": len(pats) / (t32 * 1e-3), "ms": t32, "kernel_ms": k32,
                        "fp64_ms": t64, "speedup_vs_fp64": t64 / t32,
                        **error_columns(ref, h32, e32, "mixed"), **error_columns(ref, h64, e64, "fp64")}
    # mixed-n workload with collisions
    U, r, pats = W.workload("mixed_m144")
    ref = stored_oracle("mixed_m144")
    K = gbs.build_kernel(U, r)
    for nn in range(8, 25, 2):
        gbs.autotune(nn, gbs.FP64)
        gbs.autotune(nn, gbs.MIXED)
    t64, k64, h64, e64 = timed_batch(gbs, torch, K, pats, gbs.FP64)
    t32, k32, h32, e32 = timed_batch(gbs, torch, K, pats, gbs.MIXED)
    fl = sum(model_flops(len(p)) for p in pats)
    out["mixed_m144"] = {"fp64_probs_per_s": len(pats) / (t64 * 1e-3), "fp64_ms": t64, "fp64_kernel_ms": k64,
                         "fp64_roofline": frac(fl, k64),
                         "mixed_probs_per_s": len(pats) / (t32 * 1e-3), "mixed_ms": t32,
                         **error_columns(ref, h64, e64, "fp64"), **error_columns(ref, h32, e32, "mixed"),
                         "cpu_baseline": oracle_rate(pats, U, r)}
    # large instances
    U, r, pats = W.workload("large_m900")
    ref = stored_oracle("large_m900")
    K = gbs.build_kernel(U, r)
    gbs.autotune(28, gbs.FP64)
    gbs.autotune(30, gbs.FP64)
    t64, k64, h64, e64 = timed_batch(gbs, torch, K, pats, gbs.FP64, reps=2)
    t32, k32, h32, e32 = timed_batch(gbs, torch, K, pats, gbs.MIXED, reps=2)
    fl = sum(model_flops(len(p)) for p in pats)
    out["large_m900"] = {"probs_per_s": len(pats) / (t64 * 1e-3), "ms": t64, "kernel_ms": k64,
                         "subset_terms_per_s": sum(2 ** (len(p) // 2) for p in pats) / (k64 * 1e-3),
                         "roofline": frac(fl, k64),
                         "mixed_probs_per_s": len(pats) / (t32 * 1e-3), "mixed_ms": t32,
                         **error_columns(ref, h64, e64, "fp64"), **error_columns(ref, h32, e32, "mixed"),
                         "cpu_baseline": oracle_rate(pats[:16], U, r, target_s=8.0)}
    out["large_m900"]["cpu_baseline"]["sample"] += " (16 of the 64 n=28 patterns)"
    out["bunched_m8"] = bunched(gbs, torch)
    out["serving"] = serving(gbs, torch)
    out["sampler"] = sampler(gbs, measured_peak)
    return out


def bunched(gbs, torch, reps=3):
    """M = 8, r = 1, 512 patterns of 24 photons drawn with replacement: host
    index lists take the repeated-row route chosen on the host, device index
    lists the same route chosen on the device (cost prod (c_j + 1) terms); the
    explicit matrices B_x through gbs_hafnian_batch take the subset sum (cost
    2^12 subsets). Wall time per batch, the routes' largest relative deviations
    and each route's largest error estimate (the subset sum cancels far more on
    bunched patterns)."""
    U, r, pats = W.workload("bunched_m8")
    K = gbs.build_kernel(U, r)
    idx, n, offs = gbs.pack_patterns(pats)
    b = len(pats)
    hh = np.zeros(2 * b)
    eh = np.zeros(b)
    d_idx = torch.from_numpy(idx).cuda()
    hd = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    ed = torch.zeros(b, dtype=torch.float64, device="cuda")
    Bd = torch.zeros(2 * 8 * 8, dtype=torch.float64, device="cuda")
    K.copy_B(Bd)
    Bc = Bd.cpu().numpy().view(np.complex128).reshape(8, 8)
    flat, nm, om = gbs.pack_matrices([Bc[np.ix_(x, x)] for x in pats])
    d_mat = torch.from_numpy(flat).cuda()
    hm = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    km = torch.zeros(b, dtype=torch.float64, device="cuda")

    def host_route():
        gbs.prob_batch(K, idx, n, offs, gbs.FP64, haf_out=hh, err_out=eh)

    def device_route():
        gbs.prob_batch(K, d_idx, n, offs, gbs.FP64, haf_out=hd, err_out=ed)
        torch.cuda.synchronize()

    def subset_sum():
        gbs.hafnian_batch(d_mat, nm, om, gbs.FP64, haf_out=hm, kappa_out=km)
        torch.cuda.synchronize()

    gbs.autotune(24, gbs.FP64)
    ts = {}
    for name, fn in (("repeated_row", host_route), ("device_route", device_route), ("subset_sum", subset_sum)):
        fn()
        t = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            t.append(time.perf_counter() - t0)
        ts[name] = float(np.median(t))
    a = hh[0::2] + 1j * hh[1::2]
    h = hd.cpu().numpy()
    c = h[0::2] + 1j * h[1::2]
    q = hm.cpu().numpy()
    sub = q[0::2] + 1j * q[1::2]
    return {"workload": "M=8 Haar U seed 5, r=1.0, 512 patterns of n=24 drawn with replacement, FP64",
            "repeated_row_probs_per_s": b / ts["repeated_row"], "repeated_row_ms": 1e3 * ts["repeated_row"],
            "device_route_probs_per_s": b / ts["device_route"], "device_route_ms": 1e3 * ts["device_route"],
            "subset_sum_probs_per_s": b / ts["subset_sum"], "subset_sum_ms": 1e3 * ts["subset_sum"],
            "speedup": ts["subset_sum"] / ts["repeated_row"],
            "max_rel_dev_between_routes": float(np.max(np.abs(a - c) / np.abs(a))),
            "subset_sum_max_rel_dev_vs_repeated_row": float(np.max(np.abs(sub - a) / np.abs(a))),
            "repeated_row_max_err_est": float(eh.max()),
            "subset_sum_max_err_est": float(np.max(km.cpu().numpy() * 24 * 2.0 ** -53))}


def sampler(gbs, measured_peak=None):
    """Appendix I brute-force sampler at the paper's check size (n = 4, m = 16,
    400,000 draws), Step 1 (P_n) at m = 36, and Algorithm 1 chain samples of
    12, 16 and 20 photons at m = n^2: wall time through the C ABI."""
    m, n = 16, 4
    K = gbs.build_kernel(W.haar_unitary(m, 16), np.full(m, 0.5))
    u = np.random.default_rng(2019).random(400000)
    gbs.sample_bruteforce(K, n, u[:1000])
    t0 = time.perf_counter()
    pats, total = gbs.sample_bruteforce(K, n, u)
    t_bf = time.perf_counter() - t0
    K36 = gbs.build_kernel(W.haar_unitary(36, 3), np.full(36, 0.8814))
    gbs.photon_number_dist(K36, 200)
    t0 = time.perf_counter()
    gbs.photon_number_dist(K36, 200)
    t_pn = time.perf_counter() - t0
    # Algorithm 1 chain samples in the paper's m = n^2 setting (Sec. 3.5)
    chain = {}
    for n_, reps in ((12, 5), (16, 5), (20, 3)):
        m_ = n_ * n_
        Kc = gbs.build_kernel(W.haar_unitary(m_, 40 + n_), np.full(m_, 0.8814))
        rng = np.random.default_rng(n_)
        gbs.sample_chain(Kc, n_, rng.random(n_))  # warm-up
        ts = []
        for _ in range(reps):
            uu = rng.random(n_)
            t0 = time.perf_counter()
            gbs.sample_chain(Kc, n_, uu)
            ts.append(time.perf_counter() - t0)
        chain["n%d_m%d" % (n_, m_)] = {"s_per_sample": float(np.median(ts)), "samples": reps}
    # independent samples advanced together (gbs_sample_chain_batch)
    for n_, S in ((12, 1024), (16, 256), (20, 32)):
        m_ = n_ * n_
        Kc = gbs.build_kernel(W.haar_unitary(m_, 40 + n_), np.full(m_, 0.8814))
        rng = np.random.default_rng(100 + n_)
        gbs.sample_chain_batch(Kc, n_, rng.random((S, n_)))  # warm-up
        uu = rng.random((S, n_))
        t0 = time.perf_counter()
        gbs.sample_chain_batch(Kc, n_, uu)
        dt = time.perf_counter() - t0
        fl = chain_sample_flops(n_, m_, S)
        chain["batch_n%d_m%d" % (n_, m_)] = {
            "samples": S, "s_per_batch": dt, "samples_per_s": S / dt,
            "fp64_tflops": fl / dt / 1e12, "frac_of_fp64_peak": fl / dt / 1e12 / fp64_peak_tflops(),
            "frac_of_measured_fp64_peak": (fl / dt / 1e12 / measured_peak) if measured_peak else None,
            "work_note": "chain_sample_flops: the products, row expansions and cache updates the kernels form, "
                         "8 flops per complex multiply-add; whole-call wall time"}
    return {"bruteforce_n4_m16": {"configurations": 3876, "draws": len(u), "wall_ms": 1e3 * t_bf,
                                  "draws_per_s": len(u) / t_bf, "P_n": total},
            "photon_number_m36_nmax200_wall_ms": 1e3 * t_pn,
            "chain_sampler": chain}


def serve_stream(gbs, K, reqs, precision):
    """Poisson client: submit at the scheduled arrival times, poll until done.
    Latency = completion seen by the client - scheduled arrival."""
    srv = gbs.Server(K, max_n=26)
    try:
        warm = [srv.submit(x, precision) for _, x in reqs[:64]]
        for t in warm:
            while srv.poll(t) is None:
                pass
        lat, even, outstanding, i = [], [], {}, 0
        # the client is Python: keep its cyclic garbage collector from pausing
        # it mid-stream (a pause would count as latency of every request due
        # in it); the server is native code and unaffected either way
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        while i < len(reqs) or outstanding:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i][0] <= now:
                tk = srv.submit(reqs[i][1], precision)
                if tk < 0:
                    break
                outstanding[tk] = (reqs[i][0], len(reqs[i][1]) % 2 == 0)
                i += 1
            for tk in list(outstanding):
                if srv.poll(tk) is not None:
                    arr, ev = outstanding.pop(tk)
                    lat.append(time.perf_counter() - t0 - arr)
                    even.append(ev)
        total = time.perf_counter() - t0
        st = srv.stats()
    finally:
        gc.enable()
        srv.destroy()
    lat = np.array(lat) * 1e3
    le = lat[np.array(even, dtype=bool)]  # odd n is answered at submission (p = 0)
    return {"requests": len(reqs), "throughput_req_s": len(reqs) / total, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "even_n_p50_ms": float(np.percentile(le, 50)), "even_n_p99_ms": float(np.percentile(le, 99)),
            # the server's own view: device steps, their mean and longest wall time
            # (launch to detected completion) and device time (CUDA events around
            # the step); a long wall tail over short device steps points at the host
            "steps": int(st["steps"]), "step_mean_ms": 1e3 * st["step_wall_s"] / max(1, st["steps"]),
            "step_max_ms": 1e3 * st["step_wall_max_s"],
            "step_device_mean_ms": 1e3 * st["step_device_s"] / max(1, st["steps"]),
            "step_device_max_ms": 1e3 * st["step_device_max_s"],
            # the server thread's longest pause between loop iterations or polls,
            # and its longest step launch call
            "poll_gap_max_ms": 1e3 * st["poll_gap_max_s"], "launch_max_ms": 1e3 * st["launch_max_s"],
            "update_max_ms": 1e3 * st["update_max_s"], "submit_max_ms": 1e3 * st["submit_max_s"]}


def serve_load(gbs, K, reqs, precision):
    """Open-loop Poisson client for the saturation sweep: submits at the
    scheduled arrival times (a full queue is retried) and collects finished
    requests through the completion queue (gbs_serve_wait_any), so the client
    does not poll each ticket. Latency = collection time - scheduled arrival."""
    srv = gbs.Server(K, max_n=26)
    try:
        for _, x in reqs[:64]:
            srv.submit(x, precision)
        got = 0
        while got < 64:
            got += len(srv.wait_any(0.05)[0])
        arr = np.array([a for a, _ in reqs])
        xs = [np.ascontiguousarray(x, dtype=np.int32) for _, x in reqs]
        lat = np.empty(len(reqs))
        where = {}
        i = done = 0
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and arr[i] <= now:
                tk = srv.submit(xs[i], precision)
                if tk < 0:
                    break
                where[tk] = i
                i += 1
            wait = 0.0 if i >= len(reqs) else max(0.0, min(arr[i] - now, 0.002))
            tks = srv.wait_any(wait if i < len(reqs) else 0.002)[0]
            tnow = time.perf_counter() - t0
            for tk in tks:
                lat[done] = tnow - arr[where.pop(int(tk))]
                done += 1
        total = time.perf_counter() - t0
    finally:
        gc.enable()
        srv.destroy()
    return lat, total


def saturation_summary(rate, lat, total):
    lat_ms = lat * 1e3
    q = len(lat) // 4
    return {"offered_req_s": rate, "throughput_req_s": len(lat) / total,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            # latency drift over the run: a queue that grows shows as a rising median
            "median_first_quarter_ms": float(np.median(lat_ms[:q])),
            "median_last_quarter_ms": float(np.median(lat_ms[-q:]))}


def sustainable(row):
    """Kept up: 95 % of the offered rate served, and no queue build-up (the
    last quarter's median latency under twice the first quarter's + 1 ms)."""
    return (row["throughput_req_s"] >= 0.95 * row["offered_req_s"]
            and row["median_last_quarter_ms"] <= 2.0 * row["median_first_quarter_ms"] + 1.0)


def saturation(gbs, K, dur_s=1.0, max_levels=24):
    """Rising Poisson rates (x1.25 from 1000 req/s, about dur_s of requests
    each) until the stream is no longer sustained; the largest sustained rate
    for the FP64 server, the mixed server and plain per-pattern calls."""
    out = {"criterion": "served >= 0.95 x offered and last-quarter median latency <= "
                        "2 x first-quarter median + 1 ms", "levels": {}}
    for name in ("fp64", "mixed", "per_pattern_fp64"):
        rows, best = [], None
        rate = 1000.0
        for _ in range(max_levels):
            count = int(rate * dur_s) + 64
            reqs = W.serving_requests(count, rate_hz=rate)
            if name == "per_pattern_fp64":
                lat, total = per_pattern_load(gbs, K, reqs)
            else:
                lat, total = serve_load(gbs, K, reqs, gbs.FP64 if name == "fp64" else gbs.MIXED)
            row = saturation_summary(rate, lat, total)
            row["sustained"] = sustainable(row)
            rows.append(row)
            if not row["sustained"]:
                break
            best = row
            rate *= 1.25
        out["levels"][name] = rows
        out[name + "_max_sustained_req_s"] = best["offered_req_s"] if best else None
        out[name + "_at_max"] = ({"p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"]} if best else None)
    return out


def per_pattern_load(gbs, K, reqs):
    """per_pattern_stream's client for the sweep: (latencies s, total s)."""
    p = np.zeros(1)
    for _, x in reqs[:64]:
        idx, n, offs = gbs.pack_patterns([x])
        gbs.prob_batch(K, idx, n, offs, gbs.FP64, p_out=p)
    lat = np.empty(len(reqs))
    gc.collect()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for j, (arr, x) in enumerate(reqs):
            now = time.perf_counter() - t0
            if now < arr:
                time.sleep(arr - now)
            idx, n, offs = gbs.pack_patterns([x])
            gbs.prob_batch(K, idx, n, offs, gbs.FP64, p_out=p)
            lat[j] = time.perf_counter() - t0 - arr
        total = time.perf_counter() - t0
    finally:
        gc.enable()
    return lat, total


def per_pattern_stream(gbs, K, reqs):
    """Plain FP64 per-pattern method: one synchronous gbs_prob_batch call per
    request, in arrival order (host buffers)."""
    p = np.zeros(1)
    lat = []
    for _, x in reqs[:64]:  # warm-up, as for the server: launch shapes, staging buffers
        idx, n, offs = gbs.pack_patterns([x])
        gbs.prob_batch(K, idx, n, offs, gbs.FP64, p_out=p)
    gc.collect()
    gc.disable()  # as in serve_stream: no collector pauses inside the client loop
    try:
        t0 = time.perf_counter()
        for arr, x in reqs:
            now = time.perf_counter() - t0
            if now < arr:
                time.sleep(arr - now)
            idx, n, offs = gbs.pack_patterns([x])
            gbs.prob_batch(K, idx, n, offs, gbs.FP64, p_out=p)
            lat.append(time.perf_counter() - t0 - arr)
        total = time.perf_counter() - t0
    finally:
        gc.enable()
    lat = np.array(lat) * 1e3
    le = lat[np.array([len(x) % 2 == 0 for _, x in reqs], dtype=bool)]
    return {"requests": len(reqs), "throughput_req_s": len(reqs) / total, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "even_n_p50_ms": float(np.percentile(le, 50)), "even_n_p99_ms": float(np.percentile(le, 99))}


def serving(gbs, torch, count: int = 20000):
    """M = 256, r = 0.88; Poisson 2000 req/s; n ~ U{12..26} collision-free."""
    U, r, _ = W.workload("serving_m256")
    K = gbs.build_kernel(U, r)
    reqs = W.serving_requests(count)
    out = {"workload": "M=256 Haar U seed 3, r=0.88, Poisson 2000 req/s, n~U{12..26} collision-free",
           "fp64": serve_stream(gbs, K, reqs, gbs.FP64),
           "mixed": serve_stream(gbs, K, reqs, gbs.MIXED),
           "per_pattern_fp64": per_pattern_stream(gbs, K, reqs[: max(1, count // 4)]),
           "saturation": saturation(gbs, K)}
    return out


if __name__ == "__main__":
    main()
