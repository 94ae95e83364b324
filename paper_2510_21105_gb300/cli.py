"""Run one anneal of a named workload and print a JSON summary.

    python -m paper_2510_21105_gb300.cli --config g63like [--steps K] [--seed S]
        [--field-bits 16|8] [--replicas-per-cta 4|8] [--threads 512] [--hex]

--steps limits the run to the first K temperature steps of the schedule
(used for small profiling runs); --hex prints the best configuration in the
paper's hexadecimal format.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    from . import binding as B
    from . import build as build_mod
    from . import hexconfig
    from . import workloads as wl

    p = argparse.ArgumentParser()
    p.add_argument("--config", default="g63like", choices=sorted(wl.CONFIGS))
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--seed", type=int, default=None)
    p.add_argument("--field-bits", type=int, default=0)
    p.add_argument("--replicas-per-cta", type=int, default=0)
    p.add_argument("--threads", type=int, default=0)
    p.add_argument("--variant", type=int, default=0)
    p.add_argument("--hex", action="store_true")
    a = p.parse_args(argv)
    build_mod.build()
    c = wl.CONFIGS[a.config]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    K = c["K"] if a.steps is None else min(a.steps, c["K"])
    seed = c["seed"] if a.seed is None else a.seed
    with B.Annealer.from_graph(g) as ann:
        t0 = time.perf_counter()
        ann.begin(betas, c["R"], c["S"], seed, nlm_period=c["nlm_period"], field_bits=a.field_bits,
                  replicas_per_cta=a.replicas_per_cta, threads_per_cta=a.threads, variant=a.variant)
        ann.run(K)
        ann.sync()
        dt = time.perf_counter() - t0
        st = ann.stats()
        cut, cfg, step, sweep = ann.best()
    out = dict(config=a.config, n=g.n, m=g.m, R=c["R"], S=c["S"], steps=K, seed=seed, best_cut=cut,
               best_step=step, best_sweep=sweep, wall_s=dt, attempts=st["attempts"],
               accepts=st["accepts"], device_ms=st["anneal_ms"],
               attempts_per_s=st["attempts"] / max(st["anneal_ms"], 1e-9) * 1e3)
    if a.hex:
        out["config_hex"] = hexconfig.encode(cfg)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
