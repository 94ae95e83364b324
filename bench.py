#!/usr/bin/env python3
"""Benchmark: spin-flip attempts per second of population annealing on a
G63-shaped Max-Cut instance (N = 7000, M = 41,459 unweighted random edges),
R = 16384 replicas, beta linear 0.1 -> 4.0 in K = 1000 steps, 10 sweeps per
step, Houdayer non-local moves every 50 steps (synthetic seeded graph).

One benchmark step = one whole anneal (all temperature steps: resampling,
sweeps, best tracking, non-local moves), N R S K = 1.147e12 attempts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). Under torchrun every rank anneals its own
instance (seed + rank): independent problems, no data-path collective, weak
scaling; the harness barrier and the max-over-ranks time use torch.distributed.
"""
from __future__ import annotations

import argparse
import collections
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

METRIC = "spin-flip attempts/s at N=7000 R=16384 + batched/served vs plain, bit-exact"
UNIT = "attempts/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SMS = 152
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="anneal", choices=["anneal", "batch", "serve", "oracle"],
                   help="anneal: the headline line; batch / serve: the batched and served workloads; "
                        "oracle: the oracle timing plan on the host cores")
    p.add_argument("--oracle-steps", type=int, default=100,
                   help="oracle mode: steps of the single-thread G63-shaped run")
    p.add_argument("--instances", type=int, default=64)
    p.add_argument("--streams", type=int, default=32, help="batch mode: concurrent streams")
    p.add_argument("--use-graph", type=int, default=0,
                   help="batched arm: 1 = capture the batch into one CUDA graph; 0 (default) enqueues it on the "
                        "streams directly, measured faster once graph construction is timed")
    p.add_argument("--slots", type=int, default=16, help="serve mode: concurrently running requests")
    p.add_argument("--tick", type=int, default=8, help="serve mode: temperature steps per tick")
    p.add_argument("--serve-seconds", type=float, default=3.0, help="arrival window of the served trace")
    p.add_argument("--rate", type=float, default=20.0, help="mean arrivals per second")
    p.add_argument("--config", default="g63like")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch-serve", action="store_true",
                   help="skip the batched and served measurements of the default line")
    p.add_argument("--field-bits", type=int, default=0, help="0 = auto layout")
    p.add_argument("--threads", type=int, default=0, help="threads per sweep CTA (0 = auto)")
    p.add_argument("--variant", type=int, default=2, help="0 int8 layouts, 1 multi-spin coded, 2 auto")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="approximate CPU time of the oracle sample")
    return p.parse_args()


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# ------------------------------------------------------ reference (oracle) ---
def cpu_oracle_sample(cfg_name: str, seconds: float, threads: int = 1, R: int = 16):
    """Time the oracle on a bounded sample of the benchmark workload: the same
    graph and schedule, R replicas, the first temperature steps. threads > 1
    uses the oracle's OpenMP timing build (replicas swept on that many host
    threads between resamplings; same results)."""
    import oracle
    from paper_2510_21105_gb300 import workloads as wl

    c = wl.CONFIGS[cfg_name]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    par = threads > 1
    if par:
        oracle.lib_parallel(threads)
    # calibrate: 2 steps, then scale the step count to the time budget
    t0 = time.perf_counter()
    oracle.anneal(g.rp, g.col, g.w, betas[:2], R=R, S=c["S"], seed=c["seed"], parallel=par)
    per_step = (time.perf_counter() - t0) / 2
    K = int(max(2, min(c["K"], seconds / max(per_step, 1e-6))))
    t0 = time.perf_counter()
    oracle.anneal(g.rp, g.col, g.w, betas[:K], R=R, S=c["S"], seed=c["seed"],
                  nlm_period=c["nlm_period"], parallel=par)
    dt = time.perf_counter() - t0
    attempts = g.n * R * c["S"] * K
    return {"value": attempts / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{cfg_name} graph, R={R}, first {K} of {c['K']} steps x {c['S']} sweeps "
                      f"({attempts:.3g} attempts, {dt:.1f} s, "
                      + ("single thread" if not par else f"{threads} threads, OpenMP over replicas") + ")"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_plan(args):
    """The oracle timing plan of the measurement: the small random-graph
    workload (N=800, R=256, K=100, S=4) in full, and the G63-shaped graph and
    the 100 x 100 torus with R=256 over all their steps, on one host core and on
    all of them (the single-thread runs of the latter two are bounded to
    --oracle-steps steps)."""
    import oracle
    from paper_2510_21105_gb300 import workloads as wl

    cores = host_cores()
    out = {"mode": "oracle", "unit": UNIT, "nproc": cores, "runs": []}
    for name, R, K1 in (("gnp800", 256, None), ("g63like", 256, args.oracle_steps),
                        ("torus100", 256, args.oracle_steps)):
        c = wl.CONFIGS[name]
        g = c["graph"]()
        betas = wl.linear_betas(*c["beta"], c["K"])
        for threads in (1, cores):
            K = c["K"] if (threads > 1 or K1 is None) else min(K1, c["K"])
            if threads > 1:
                oracle.lib_parallel(threads)
            t0 = time.perf_counter()
            res = oracle.anneal(g.rp, g.col, g.w, betas[:K], R=R, S=c["S"], seed=c["seed"],
                                nlm_period=c["nlm_period"], parallel=threads > 1)
            dt = time.perf_counter() - t0
            att = g.n * R * c["S"] * K
            out["runs"].append({"workload": name, "R": R, "steps": K, "of_steps": c["K"], "threads": threads,
                                "attempts": att, "seconds": dt, "attempts_per_s": att / dt,
                                "best_cut": int((oracle.total_weight(g.rp, g.col, g.w) - res.best_E) // 2)})
            print(json.dumps(out["runs"][-1]), flush=True)
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2510_21105_gb300 import workloads as wl

    c = wl.CONFIGS[args.config]
    samples = []
    for _ in range(args.warmup):
        cpu_oracle_sample(args.config, min(args.cpu_seconds, 3.0))
    for _ in range(args.steps):
        samples.append(cpu_oracle_sample(args.config, args.cpu_seconds))
    v = statistics.median(s["value"] for s in samples)
    ms = 1000.0 * (wl.CONFIGS[args.config]["graph"]().n * c["R"] * c["S"] * c["K"]) / v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{args.config}: N=7000 M=41459 R={c['R']} K={c['K']} S={c['S']} "
                                   f"nlm_period={c['nlm_period']}", "l2": "n/a (CPU)"},
            "cpu_baseline": {**samples[-1], "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours ---
# DRAM bytes (read + write) of one sweep step on this workload (the head and
# tail launches of the multi-spin-coded sweep, or the one launch of another
# layout), from one ncu capture, with the SHA-256 prefix of the sweep source it
# was taken on: reported only while that source is the one that runs.
SWEEP_TRAFFIC = {"k_sweep_msc+pair": ((102.875648 + 44.824064 + 12.869376) * 1e6, "6ca9288e529d8511")}
SWEEP_SRC = os.path.join(ROOT, "paper_2510_21105_gb300", "csrc", "k_sweep.cu")
INT_LANES_PER_SM = 128   # ALU pipe 64 + FMA pipe 64 integer lanes per SM and clock (unit counts)
SMEM_BYTES_PER_SM = 128  # shared-memory bytes per SM and clock (32 banks x 4 B)


def sweep_source_sha() -> str:
    import hashlib

    with open(SWEEP_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def msc_planes(max_degree: int) -> int:
    """Bit planes of the frustrated-bond counters (counts up to max_degree)."""
    return 3 if max_degree <= 7 else 4 if max_degree <= 15 else 5 if max_degree <= 31 else 6 if max_degree <= 63 else 7


def msc_ops_per_attempt(mean_degree: float, max_degree: int = 31) -> float:
    """Algorithmic integer instructions of one multi-spin-coded attempt: one
    item (one position of a 32-replica word) divided by its 32 attempts.
      bond counting   per 4 bonds, three-input logic ops of the carry-save
                      adders: 7 + 2 (NPL - 3) with the planes kept
                      complemented (NPL >= 4), 13 with plain adders from
                      zero (NPL = 3); NPL ops to decode the complemented form
      count bytes     8 x 8 bit transpose in every byte lane: 12 swaps x 4 ops
      uniforms        2 Philox4x32-10 calls x 10 rounds x (2 widening
                      multiplies + 2 three-input xors)
      decisions       per 4-replica group: 2 pair-table offsets (dot products),
                      2 uniform spreads, 2 multiply-adds, 2 subtracts, 2 sign
                      permutes, 2 mask merges (NPL <= 5; wider counts: 4 index
                      extracts and 2 half-word merges instead of the offsets)
      energies        per group: table index, count byte, masked select, add
    Loads, addressing, loop control, barriers and the row packing at load and
    store are not counted."""
    npl = msc_planes(max_degree)
    if npl >= 4:
        bonds = (7 + 2 * (npl - 3)) / 4.0 * mean_degree + npl
    else:
        bonds = 13 / 4.0 * mean_degree
    decisions = 8 * (12 if npl <= 5 else 16)
    per_item = bonds + 12 * 4 + 2 * 10 * 4 + decisions + 8 * 4
    return per_item / 32.0


def packed_ops_per_attempt(mean_degree: float, accept_rate: float) -> float:
    """4-replica layouts: one Philox call per 4 attempts (40 ops), the
    decision (5) and the field updates of an accepted flip (2 per bond)."""
    return 40.0 / 4 + 5.0 + accept_rate * 2.0 * mean_degree


def smem_bytes_per_attempt(kernel, mean_degree, accept_rate):
    """Algorithmic shared-memory bytes of one attempt. Multi-spin coded (the
    measurement plan's figure): (8 + 6 d) / 32, the item's own word read and
    written plus a 4-byte neighbour word and its 2-byte index per bond, over
    32 attempts. 4-replica layouts: the spin/field byte read and written and
    the threshold word, plus the neighbours' field bytes read and written on
    an accepted flip."""
    if kernel[0].startswith("k_sweep_msc"):
        return (8.0 + 6.0 * mean_degree) / 32.0
    return 2.0 + 4.0 + accept_rate * 2.0 * mean_degree


def sweep_roofline(stats, attempts_per_launch, probe, clk_mhz, kernel, mean_degree, accept_rate, sms=SMS,
                   max_degree=31):
    """Roofline of the sweep (the dominant kernel): integer-issue bound.
    probe: pa_probe_peaks of the device (measured peaks) or None."""
    launches = max(stats["sweep_launches"], 1)
    t = stats["sweep_ms"] / launches / 1e3
    if t <= 0:
        return None
    aps = attempts_per_launch / t
    msc = kernel[0].startswith("k_sweep_msc")
    ops = msc_ops_per_attempt(mean_degree, max_degree) if msc else packed_ops_per_attempt(mean_degree, accept_rate)
    achieved = aps * ops / 1e12
    derived = sms * INT_LANES_PER_SM * clk_mhz * 1e6 / 1e12
    peak = probe["int_ops_per_s"] / 1e12 if probe else derived
    sbpa = smem_bytes_per_attempt(kernel, mean_degree, accept_rate)
    smem_derived = sms * SMEM_BYTES_PER_SM * clk_mhz * 1e6
    smem_peak = probe["smem_bytes_per_s"] if probe else smem_derived
    traffic = SWEEP_TRAFFIC.get(kernel[0])
    if traffic and traffic[1] != sweep_source_sha():
        traffic = None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": traffic[0] if traffic else None,
            "kernel": f"{kernel[0]}<{kernel[1]} threads>", "avg_launch_ms": t * 1e3,
            "attempts_per_s_in_kernel": aps, "ops_per_attempt": ops,
            "peak_source": ("measured on this GPU by pa_probe_peaks (1:1 IMAD + LOP3 integer instructions)"
                            if probe else f"derived: {sms} SMs x {INT_LANES_PER_SM} integer lanes x {clk_mhz:.0f} MHz"),
            "peak_derived": derived, "frac_vs_derived": achieved / derived,
            "smem_bytes_per_attempt": sbpa, "smem_frac": aps * sbpa / smem_peak,
            "smem_frac_vs_derived": aps * sbpa / smem_derived,
            "smem_target_met": aps * sbpa / smem_peak >= 0.5,
            "philox_frac": (aps * (0.25 if msc else 1.0) / probe["philox_words_per_s"]) if probe else None,
            # The same rate against the count of the first formulation (plain carry-save adders, one table lookup
            # per replica: (4.5 d + 288)/32), which stays fixed across builds and so tracks the kernel's progress.
            "ops_per_attempt_first_formulation": (4.5 * mean_degree + 288.0) / 32.0 if msc else None,
            "frac_first_formulation": aps * (4.5 * mean_degree + 288.0) / 32.0 / 1e12 / peak if msc else None}


def max_over_ranks(x: float, dist, device: str = "cpu") -> float:
    """The slowest rank's time (every rank anneals its own instance)."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(attempts_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job attempts per second: all ranks' attempts over the slowest rank's time."""
    return world * attempts_per_rank / (ms_max / 1e3)


def run_ours(args, rank, world, dist):
    import torch

    from paper_2510_21105_gb300 import binding as B
    from paper_2510_21105_gb300 import build as build_mod
    from paper_2510_21105_gb300 import workloads as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        build_mod.build()
    if dist:
        dist.barrier()
    B.lib()
    c = wl.CONFIGS[args.config]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    R, S, K = c["R"], c["S"], c["K"]
    seed = c["seed"] + rank
    stream = torch.cuda.current_stream()
    sh = B.C.c_void_p(stream.cuda_stream)
    attempts = g.n * R * S * K

    ann = B.Annealer.from_graph(g)

    def one(time_kernels=0):
        ann.anneal(betas, R, S, seed, nlm_period=c["nlm_period"], stream=sh,
                   time_kernels=time_kernels, field_bits=args.field_bits,
                   threads_per_cta=args.threads, variant=args.variant)

    for _ in range(args.warmup):
        one()
    variant_run = ann.stats()["variant"]
    if variant_run == 1:
        layout, kernel = "multi-spin coded (32 replicas per 32-bit word)", ("k_sweep_msc", args.threads or 256)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        words = (R + 31) // 32
        if words > sms and words % sms:
            layout += f"; {words // sms * sms} words in one-CTA blocks + {words % sms} in CTA pairs, concurrently"
            kernel = ("k_sweep_msc+pair", args.threads or 256)
    elif variant_run == 3:
        layout = "multi-spin coded, a cluster of two CTAs per 32-replica word"
        kernel = ("k_sweep_msc_pair", 256)
    else:
        fb = args.field_bits if args.field_bits else (7 if g.maxdeg <= 127 else 16)
        layout = {7: "packed byte (spin bit + 7-bit field)", 8: "int8 spin + int8 field",
                  16: "int8 spin + int16 field"}[fb]
        kernel = ("k_sweep_packed" if fb == 7 else "k_sweep", args.threads or (128 if fb == 7 else 512))
    peaks, peaks_src = load_peaks()
    probe = B.probe_peaks(sh)   # integer, Philox and shared-memory peaks of this GPU (a few ms)
    # timed region: device-resident inputs, K anneals
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats_acc = {"sweep_ms": 0.0, "sweep_launches": 0, "kernel_launches": 0}
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            one(time_kernels=1)
            st = ann.stats()
            for key in stats_acc:
                stats_acc[key] += st[key]
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    t_best = st["t_best_ms"]
    acc_rate = st["accepts"] / max(st["attempts"], 1)
    cut, _, best_step, _ = ann.best()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = aggregate_value(attempts, world, ms_max)
    clocks = clk.summary()
    clk_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roof = sweep_roofline(stats_acc, g.n * R * S, probe, clk_mhz, kernel, 2.0 * g.m / g.n, acc_rate,
                          sms=probe["sms"], max_degree=int(g.maxdeg))
    ann.close()

    # end to end through the C-ABI with host buffers (pinned), copies inside the region
    e2e = None
    if not args.no_e2e:
        rp = torch.from_numpy(g.rp_u32).pin_memory()
        col = torch.from_numpy(g.col_u16.view(np.int16)).pin_memory()
        hb = torch.from_numpy(betas).pin_memory()
        cfg = torch.empty(g.n, dtype=torch.int8).pin_memory()
        lib = B.lib()
        times, h2d, d2h = [], 0, 0
        for it in range(args.steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = B.C.c_void_p()
            rc = lib.pa_create(B.C.byref(ctx), g.n, rp.data_ptr(), col.data_ptr(), None)
            assert rc == 0, rc
            o = B.pa_default_opts(nlm_period=c["nlm_period"], stream=sh, field_bits=args.field_bits,
                                  threads_per_cta=args.threads, variant=args.variant)
            rc = lib.pa_anneal(ctx, hb.data_ptr(), K, R, S, seed, B.C.byref(o))
            assert rc == 0, rc
            cutv = B.C.c_int64()
            rc = lib.pa_best(ctx, B.C.byref(cutv), cfg.data_ptr(), None, None)
            assert rc == 0, rc
            st2 = B.pa_stats(ctx)
            lib.pa_destroy(ctx)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if it > 0:   # the first call pays the context's one-time set-up
                times.append(dt)
                h2d, d2h = st2["h2d_bytes"], st2["d2h_bytes"]
        e2e_s = max_over_ranks(max(statistics.median(times), 1e-9), dist, "cuda")
        e2e = {"value": world * attempts / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3}

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_sample(args.config, args.cpu_seconds)
        cores = host_cores()
        cpu["nproc"] = cores
        if cores > 1:
            allc = cpu_oracle_sample(args.config, args.cpu_seconds, threads=cores, R=256)
            cpu["all_cores"] = {k: allc[k] for k in ("value", "cores", "sample")}
    batched = served = None
    if world == 1 and not args.no_batch_serve:
        b = batch_measure(args)
        batched = {k: b[k] for k in ("ratio", "ratio_vs_default_plain", "value", "plain_value", "batch_s", "plain_s",
                                     "graph_build_and_setup_ms", "bit_identical_to_plain", "instances")}
        sv = serve_measure(args)
        served = {k: sv[k] for k in ("ratio", "value", "plain_value", "p50_ms", "p99_ms", "plain_p50_ms",
                                     "plain_p99_ms", "requests", "bit_identical_to_plain")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8/bit spins, int32 energies, fp64 weights",
            "data": "synthetic",
            "config": {"workload": f"{args.config}: G63-shaped N={g.n} M={g.m} R={R} K={K} S={S} "
                                   f"beta {c['beta'][0]}->{c['beta'][1]} nlm_period={c['nlm_period']}",
                       "l2": "inputs larger than L2 (population 688 MB per buffer pair)",
                       "seed": c["seed"]},
            "layout": layout,
            "accept_rate": acc_rate,
            "best_cut": int(cut), "best_step": int(best_step), "time_to_best_ms": t_best,
            "e2e": e2e, "gpu_launches": stats_acc["kernel_launches"],
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "peaks": peaks_src,
            "batched": batched, "served": served}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- batched ---
def batch_measure(args, reps: int = 2):
    """64 mixed instances (N ~ U[800, 20000]; random p = 12/(N-1), signed torus,
    Delaunay; R cycling 1024/4096/16384), beta 0.1 -> 3.0 in 200 steps, 4 sweeps:
    each instance annealed alone in turn (plain) vs all in one batched launch
    captured in a CUDA graph; kernel shapes from the autotuner. Both arms are
    timed the same way: host wall-clock from the first population set-up to
    the last result read back (graph capture and instantiation included in the
    batched arm, and also reported on their own)."""
    import tempfile

    import torch

    from paper_2510_21105_gb300 import autotune
    from paper_2510_21105_gb300 import binding as B
    from paper_2510_21105_gb300 import workloads as wl

    K, S = 200, 4
    betas = wl.linear_betas(0.1, 3.0, K)
    inst = wl.batch_instances(args.instances, seed=0)
    cache = os.path.join(tempfile.gettempdir(), "pa_autotune_cache.json")
    t0 = time.perf_counter()
    opts, opts_b = [], []
    cand = [c for c in autotune.CANDIDATES if c.get("variant") in (1, 3) or c.get("field_bits") == 7]
    for it in inst:
        g = it["graph"]
        o, _ = autotune.tune(g, betas, it["R"], S, seed=it["seed"], steps=1, cache_path=cache, candidates=cand)
        ob, _ = autotune.tune(g, betas, it["R"], S, seed=it["seed"], steps=1, cache_path=cache,
                              candidates=cand, context="saturated")
        opts.append(o)
        opts_b.append(ob)
    tune_s = time.perf_counter() - t0
    attempts = sum(it["graph"].n * it["R"] * S * K for it in inst)
    anns = [B.Annealer.from_graph(it["graph"]) for it in inst]

    def plain(option_list):
        torch.cuda.synchronize()
        t = time.perf_counter()
        best = []
        for ann, it, o in zip(anns, inst, option_list):
            ann.anneal(betas, it["R"], S, it["seed"], **o)
            best.append(ann.best_record())
        torch.cuda.synchronize()
        return time.perf_counter() - t, best

    anns[0].anneal(betas, inst[0]["R"], S, inst[0]["seed"], **opts[0])   # warm-up
    plain_s, plain_best = plain(opts)
    plain_default_s, _ = plain([{} for _ in inst])
    items = [(ann, betas, it["R"], S, it["seed"], K, o) for ann, it, o in zip(anns, inst, opts_b)]

    def batched():
        torch.cuda.synchronize()
        t = time.perf_counter()
        dev_ms = B.pa_batch_anneal(items, n_streams=args.streams, use_graph=bool(args.use_graph))
        best = [ann.best_record() for ann in anns]
        torch.cuda.synchronize()
        return time.perf_counter() - t, dev_ms, best

    batched()   # warm-up
    runs = [batched() for _ in range(max(reps, 1))]
    batch_s = statistics.median(r[0] for r in runs)
    dev_ms = statistics.median(r[1] for r in runs)
    same = all(b == p for b, p in zip(runs[-1][2], plain_best))
    for a in anns:
        a.close()
    return {"value": attempts / batch_s, "plain_value": attempts / plain_s, "ratio": plain_s / batch_s,
            "plain_default_value": attempts / plain_default_s, "ratio_vs_default_plain": plain_default_s / batch_s,
            "batch_s": batch_s, "plain_s": plain_s, "plain_default_s": plain_default_s,
            "batch_device_ms": dev_ms, "graph_build_and_setup_ms": batch_s * 1e3 - dev_ms,
            "bit_identical_to_plain": same, "instances": len(inst), "attempts": attempts, "autotune_s": tune_s,
            "layouts_plain": dict(collections.Counter(json.dumps(o, sort_keys=True) for o in opts)),
            "layouts_batched": dict(collections.Counter(json.dumps(o, sort_keys=True) for o in opts_b))}


def run_batch(args):
    from paper_2510_21105_gb300 import build as build_mod
    import torch

    build_mod.build()
    torch.cuda.set_device(0)
    r = batch_measure(args, reps=args.steps)
    line = {"mode": "batch", "metric": "batched attempts/s (64 mixed instances) vs plain one-instance-per-launch",
            "unit": UNIT, **r,
            "config": {"workload": "N~U[800,20000] random(p=12/(N-1))/torus/Delaunay, R 1024/4096/16384, "
                                   "beta 0.1->3.0 K=200 S=4", "n_streams": args.streams,
                       "timing": "host wall-clock, first set-up to last result, both arms"}}
    line["config"]["use_graph"] = bool(args.use_graph)
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- served ---
def _serve_trace(seconds, rate, seed=1):
    """Poisson arrivals; requests on random (p = 12/(N-1)) or signed torus
    graphs, N ~ U[800, 20000], R = round(2^U[10, 15]), beta 0.1 -> 3.0 in 200
    steps, 4 sweeps. A pool of 24 graphs is generated up front."""
    from paper_2510_21105_gb300 import workloads as wl

    rng = np.random.Generator(np.random.PCG64(seed))
    pool = []
    for t in range(24):
        n = int(rng.integers(800, 20001))
        pool.append(wl.gnp_sparse(n, 12.0 / (n - 1), seed=5000 + t) if t % 2 == 0
                    else wl.torus(int(round(np.sqrt(n))), seed=5000 + t))
    trace, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > seconds:
            break
        trace.append((t, pool[int(rng.integers(0, len(pool)))], int(round(2 ** rng.uniform(10, 15))),
                      len(trace)))
    return trace


def _serve(trace, betas, slots, saturated, steps_per_tick=8):
    """Every request asks for the automatic layout. The server gives a request
    admitted while others run the cheapest attempt on a shared device
    (multi-spin coded, every word in one-CTA blocks) and one admitted alone the
    single-instance choice; with one slot (the plain arm) every request runs
    alone. saturated only labels the arm."""
    from paper_2510_21105_gb300 import binding as B

    with B.Server(200 << 30, n_streams=slots, steps_per_tick=steps_per_tick) as srv:
        ids = []
        t0 = time.perf_counter()
        for at, g, R, seed in trace:
            delay = at - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(g, betas, R, 4, seed, variant=2))
        res = {}
        while len(res) < len(ids):
            for rid in ids:
                if rid not in res and srv.poll(rid) not in (0, 1):
                    res[rid] = srv.result(rid, config=False)
            time.sleep(0.002)
        makespan = time.perf_counter() - t0
    out = [res[r] for r in ids]
    lat = np.array([r["finish_ms"] - r["submit_ms"] for r in out])
    att = sum(r["attempts"] for r in out)
    return dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                attempts_per_s=att / makespan, makespan_s=makespan,
                best=[(r["energy"], r["step"], r["sweep"], r["slot"]) for r in out])


def serve_measure(args):
    """Served trace with continuous batching (16 slots) against the same trace
    served one request at a time."""
    from paper_2510_21105_gb300 import workloads as wl

    betas = wl.linear_betas(0.1, 3.0, 200)
    trace = _serve_trace(args.serve_seconds, args.rate)
    served = _serve(trace, betas, slots=args.slots, saturated=True, steps_per_tick=args.tick)
    plain = _serve(trace, betas, slots=1, saturated=False)
    return {"value": served["attempts_per_s"], "plain_value": plain["attempts_per_s"],
            "ratio": served["attempts_per_s"] / plain["attempts_per_s"],
            "p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"],
            "plain_p50_ms": plain["p50_ms"], "plain_p99_ms": plain["p99_ms"],
            "requests": len(trace), "bit_identical_to_plain": served["best"] == plain["best"]}


def run_serve(args):
    import torch

    from paper_2510_21105_gb300 import build as build_mod

    build_mod.build()
    torch.cuda.set_device(0)
    r = serve_measure(args)
    line = {"mode": "serve", "metric": "served attempts/s with continuous batching vs plain one-at-a-time",
            "unit": UNIT, **r,
            "config": {"workload": f"Poisson {args.rate}/s over {args.serve_seconds} s; random/torus N~U[800,20000]; "
                                   "R=round(2^U[10,15]); beta 0.1->3.0 K=200 S=4", "slots": args.slots,
                       "hbm_budget_gb": 200, "steps_per_tick": args.tick}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "oracle":
        return run_oracle_plan(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist

        backend = "nccl" if (torch.cuda.is_available() and args.impl == "ours") else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group(backend)
        dist = tdist
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_ours(args, rank, world, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
