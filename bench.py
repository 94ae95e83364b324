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
    p.add_argument("--mode", default="anneal", choices=["anneal", "batch", "serve"],
                   help="anneal: the headline line; batch / serve: the batched and served workloads")
    p.add_argument("--instances", type=int, default=64)
    p.add_argument("--streams", type=int, default=32, help="batch mode: concurrent streams")
    p.add_argument("--serve-seconds", type=float, default=3.0, help="arrival window of the served trace")
    p.add_argument("--rate", type=float, default=20.0, help="mean arrivals per second")
    p.add_argument("--config", default="g63like")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
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
def cpu_oracle_sample(cfg_name: str, seconds: float):
    """Time the oracle on a bounded sample of the benchmark workload: the same
    graph and schedule, a few replicas, the first temperature steps."""
    import oracle
    from paper_2510_21105_gb300 import workloads as wl

    c = wl.CONFIGS[cfg_name]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    R = 16
    # calibrate: 2 steps, then scale the step count to the time budget
    t0 = time.perf_counter()
    oracle.anneal(g.rp, g.col, g.w, betas[:2], R=R, S=c["S"], seed=c["seed"])
    per_step = (time.perf_counter() - t0) / 2
    K = int(max(2, min(c["K"], seconds / max(per_step, 1e-6))))
    t0 = time.perf_counter()
    oracle.anneal(g.rp, g.col, g.w, betas[:K], R=R, S=c["S"], seed=c["seed"],
                  nlm_period=c["nlm_period"])
    dt = time.perf_counter() - t0
    attempts = g.n * R * c["S"] * K
    return {"value": attempts / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{cfg_name} graph, R={R}, first {K} of {c['K']} steps x {c['S']} sweeps "
                      f"({attempts:.3g} attempts, {dt:.1f} s, single thread)"}


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
# DRAM bytes (read + write) of one sweep launch on this workload, from one ncu
# capture of the kernel; reported only while the captured kernel is the one
# that runs. The multi-spin-coded kernels changed after their last capture, so
# they report none.
SWEEP_TRAFFIC = {("k_sweep_packed", 128): 334.719744e6 + 289.454080e6}
OPS_PER_ATTEMPT = 20.0   # a quarter Philox4x32-10 block (15) + decision (4) + flip updates (~1)
INT_LANES_PER_SM = 128   # ALU pipe (LOP3/IADD3) 64 + FMA pipe (IMAD) 64


def smem_bytes_per_attempt(kernel, mean_degree, accept_rate):
    """Algorithmic shared-memory bytes of one attempt. Multi-spin coded: per
    (position, 32-replica word) item the neighbours' words and the item's own
    word read and written, spread over 32 attempts, plus the two 4-byte halves
    of the decision-table entry of each attempt. 4-replica layouts: the
    spin/field byte read and written and the threshold word, plus the
    neighbours' field bytes read and written on an accepted flip."""
    if kernel[0].startswith("k_sweep_msc"):
        return (4.0 * mean_degree + 8.0) / 32.0 + 8.0
    return 2.0 + 4.0 + accept_rate * 2.0 * mean_degree


def sweep_roofline(stats, attempts_per_launch, peaks, kernel, mean_degree, accept_rate):
    """Roofline of the sweep kernel (dominant kernel): integer-issue bound."""
    launches = max(stats["sweep_launches"], 1)
    t = stats["sweep_ms"] / launches / 1e3
    if t <= 0:
        return None
    achieved = attempts_per_launch * OPS_PER_ATTEMPT / t / 1e12
    clk = peaks.get("sm_max_mhz", 2070.0)
    peak = SMS * INT_LANES_PER_SM * clk * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": SWEEP_TRAFFIC.get(kernel),
            "kernel": f"{kernel[0]}<{kernel[1]} threads>", "avg_launch_ms": t * 1e3,
            "attempts_per_s_in_kernel": attempts_per_launch / t,
            "peak_source": f"derived: {SMS} SMs x {INT_LANES_PER_SM} integer lanes x {clk:.0f} MHz",
            "smem_bytes_per_attempt": smem_bytes_per_attempt(kernel, mean_degree, accept_rate),
            "smem_frac": attempts_per_launch * smem_bytes_per_attempt(kernel, mean_degree, accept_rate) / t
                         / (SMS * 128 * clk * 1e6)}


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
    roof = sweep_roofline(stats_acc, g.n * R * S, peaks, kernel, 2.0 * g.m / g.n, acc_rate)
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
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "peaks": peaks_src}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- batched ---
def run_batch(args):
    """64 mixed instances (N ~ U[800, 20000]; random p = 12/(N-1), signed torus,
    Delaunay; R cycling 1024/4096/16384), beta 0.1 -> 3.0 in 200 steps, 4 sweeps:
    each instance annealed alone in turn (plain) vs all in one batched launch
    captured in a CUDA graph; kernel shapes from the autotuner."""
    import tempfile

    import torch

    from paper_2510_21105_gb300 import autotune
    from paper_2510_21105_gb300 import binding as B
    from paper_2510_21105_gb300 import build as build_mod
    from paper_2510_21105_gb300 import workloads as wl

    build_mod.build()
    torch.cuda.set_device(0)
    K, S = 200, 4
    betas = wl.linear_betas(0.1, 3.0, K)
    inst = wl.batch_instances(args.instances, seed=0)
    cache = os.path.join(tempfile.gettempdir(), "pa_autotune_cache.json")
    t0 = time.perf_counter()
    opts, opts_b = [], []
    cand = [c for c in autotune.CANDIDATES if c.get("variant") in (1, 3) or c.get("field_bits") == 7]
    for i, it in enumerate(inst):
        g = it["graph"]
        o, _ = autotune.tune(g, betas, it["R"], S, seed=it["seed"], steps=1, cache_path=cache, candidates=cand)
        ob, _ = autotune.tune(g, betas, it["R"], S, seed=it["seed"], steps=1, cache_path=cache,
                              candidates=cand, context="saturated")
        opts.append(o)
        opts_b.append(ob)
    tune_s = time.perf_counter() - t0
    attempts = sum(it["graph"].n * it["R"] * S * K for it in inst)
    anns = [B.Annealer.from_graph(it["graph"]) for it in inst]
    # plain: one instance after another, each its own pa_anneal
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ann0 = anns[0]
    ann0.anneal(betas, inst[0]["R"], S, inst[0]["seed"], **opts[0])   # warm-up
    torch.cuda.synchronize()
    ev0.record()
    plain_best = []
    for ann, it, o in zip(anns, inst, opts):
        ann.anneal(betas, it["R"], S, it["seed"], **o)
        plain_best.append(ann.best_record())
    ev1.record()
    torch.cuda.synchronize()
    plain_ms = ev0.elapsed_time(ev1)
    # plain with the library's default layout choice (no per-instance tuning)
    ev0.record()
    for ann, it in zip(anns, inst):
        ann.anneal(betas, it["R"], S, it["seed"])
    ev1.record()
    torch.cuda.synchronize()
    plain_default_ms = ev0.elapsed_time(ev1)
    items = [(ann, betas, it["R"], S, it["seed"], K, o) for ann, it, o in zip(anns, inst, opts_b)]
    B.pa_batch_anneal(items, n_streams=args.streams, use_graph=True)   # warm-up (and graph build)
    times = [B.pa_batch_anneal(items, n_streams=args.streams, use_graph=True) for _ in range(max(args.steps, 1))]
    batch_ms = statistics.median(times)
    same = all(ann.best_record() == b for ann, b in zip(anns, plain_best))
    for a in anns:
        a.close()
    line = {"mode": "batch", "metric": "batched attempts/s (64 mixed instances) vs plain one-instance-per-launch",
            "value": attempts / (batch_ms / 1e3), "unit": UNIT, "plain_value": attempts / (plain_ms / 1e3),
            "ratio": plain_ms / batch_ms, "batch_ms": batch_ms, "plain_ms": plain_ms,
            "plain_default_value": attempts / (plain_default_ms / 1e3), "plain_default_ms": plain_default_ms,
            "ratio_vs_default_plain": plain_default_ms / batch_ms,
            "bit_identical_to_plain": same, "instances": len(inst), "attempts": attempts,
            "autotune_s": tune_s,
            "layouts_plain": dict(collections.Counter(json.dumps(o, sort_keys=True) for o in opts)),
            "layouts_batched": dict(collections.Counter(json.dumps(o, sort_keys=True) for o in opts_b)),
            "config": {"workload": "N~U[800,20000] random(p=12/(N-1))/torus/Delaunay, R 1024/4096/16384, "
                                   "beta 0.1->3.0 K=200 S=4", "use_graph": True, "n_streams": args.streams}}
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


def _serve(trace, betas, slots, saturated):
    """saturated: other requests keep the GPU full, so each request uses the
    kernel with the cheapest attempt (multi-spin coded); otherwise each uses
    the automatic choice for a GPU of its own."""
    from paper_2510_21105_gb300 import binding as B

    with B.Server(200 << 30, n_streams=slots, steps_per_tick=8) as srv:
        ids = []
        t0 = time.perf_counter()
        for at, g, R, seed in trace:
            delay = at - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            variant = 1 if (saturated and g.maxdeg <= 127) else 2
            ids.append(srv.submit(g, betas, R, 4, seed, variant=variant))
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


def run_serve(args):
    import torch

    from paper_2510_21105_gb300 import build as build_mod
    from paper_2510_21105_gb300 import workloads as wl

    build_mod.build()
    torch.cuda.set_device(0)
    betas = wl.linear_betas(0.1, 3.0, 200)
    trace = _serve_trace(args.serve_seconds, args.rate)
    served = _serve(trace, betas, slots=16, saturated=True)
    plain = _serve(trace, betas, slots=1, saturated=False)
    line = {"mode": "serve", "metric": "served attempts/s with continuous batching vs plain one-at-a-time",
            "value": served["attempts_per_s"], "unit": UNIT, "plain_value": plain["attempts_per_s"],
            "ratio": served["attempts_per_s"] / plain["attempts_per_s"],
            "p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"],
            "plain_p50_ms": plain["p50_ms"], "plain_p99_ms": plain["p99_ms"],
            "requests": len(trace), "bit_identical_to_plain": served["best"] == plain["best"],
            "config": {"workload": f"Poisson {args.rate}/s over {args.serve_seconds} s; random/torus N~U[800,20000]; "
                                   "R=round(2^U[10,15]); beta 0.1->3.0 K=200 S=4", "slots": 16,
                       "hbm_budget_gb": 200, "steps_per_tick": 8}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
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
