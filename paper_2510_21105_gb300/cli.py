"""Command line: anneal a named workload or a G-set file, or verify a cut.

    python -m paper_2510_21105_gb300.cli [--config g63like | --graph FILE]
        [--steps K] [--seed S] [--replicas R] [--sweeps S] [--beta LO HI K]
        [--nlm-period P] [--nlm-kind 0|1] [--nlm-block B] [--variant 0|1|2|3] [--field-bits 16|8|7]
        [--replicas-per-cta 4|8] [--threads T] [--hex] [--save-hex FILE]
        [--curve FILE] [--checkpoint FILE --checkpoint-every K] [--resume FILE]
        [--adaptive 1|2 [--rho F] [--adapt-J J] [--dbeta-max D] [--beta-max B] [--acc-lo F --acc-hi F]]
        [--reheat-after Q --reheat-back N]

    python -m paper_2510_21105_gb300.cli verify --graph FILE --hex-file FILE
        [--expect-cut C]

The first form runs one anneal and prints a JSON summary; --steps limits the
run to the first K temperature steps of the schedule (used for small
profiling runs); --hex prints the best configuration in the paper's
hexadecimal format (Sec. 3) and --save-hex writes it to a file. A --graph
file is in the G-set text format ("n m", then "i j w" per edge, 1-based);
its schedule defaults to R=16384, S=10, beta 0.1 -> 4.0 over K=1000 steps,
non-local moves every 50 steps.

--adaptive 1 chooses each temperature step by the ESS rule, --adaptive 2
by the acceptance-rate rule (both on the grid of --dbeta-max / 2^J up to
--beta-max, with --steps / K as the cap), and --reheat-after steps back the
fixed schedule after that many steps without a lower energy (the adaptive
control options of pa_anneal_opts).

For long runs, --checkpoint/--checkpoint-every save the whole anneal every K
steps and --resume continues one (bit-exact: all randomness is counter based,
so a resumed run equals an uninterrupted one). --curve writes the best cut
so far at the end of every step with its device time (cut-vs-time curve).

The verify form evaluates the cut of a hexadecimal configuration on the
given graph on the device (pa_energies) and exits 1 if --expect-cut is given
and differs.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

DEFAULT_FILE_SCHEDULE = dict(R=16384, S=10, beta=(0.1, 4.0), K=1000, nlm_period=50, seed=0)


def _verify(argv):
    from . import binding as B
    from . import build as build_mod
    from . import hexconfig
    from . import workloads as wl

    p = argparse.ArgumentParser(prog="cli verify")
    p.add_argument("--graph", required=True)
    p.add_argument("--hex-file", required=True)
    p.add_argument("--expect-cut", type=int, default=None)
    a = p.parse_args(argv)
    build_mod.build()
    g = wl.read_gset(a.graph)
    with open(a.hex_file) as f:
        text = "".join(line.split("#", 1)[0] for line in f)
    x = hexconfig.decode(text, g.n)
    with B.Annealer.from_graph(g) as ann:
        E, cuts = ann.energies(x)
    out = dict(graph=a.graph, n=g.n, m=g.m, energy=int(E[0]), cut=int(cuts[0]))
    ok = a.expect_cut is None or int(cuts[0]) == a.expect_cut
    if a.expect_cut is not None:
        out["expected_cut"] = a.expect_cut
        out["match"] = ok
    print(json.dumps(out))
    return 0 if ok else 1


def _anneal(argv):
    from . import binding as B
    from . import build as build_mod
    from . import hexconfig
    from . import workloads as wl

    p = argparse.ArgumentParser()
    src = p.add_mutually_exclusive_group()
    src.add_argument("--config", default=None, choices=sorted(wl.CONFIGS))
    src.add_argument("--graph", default=None)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--seed", type=int, default=None)
    p.add_argument("--replicas", type=int, default=None)
    p.add_argument("--sweeps", type=int, default=None)
    p.add_argument("--beta", type=float, nargs=3, metavar=("LO", "HI", "K"), default=None)
    p.add_argument("--nlm-period", type=int, default=None)
    p.add_argument("--nlm-kind", type=int, default=0, help="0 Houdayer pairs, 1 block moves")
    p.add_argument("--nlm-block", type=int, default=32, help="block move size")
    p.add_argument("--field-bits", type=int, default=0)
    p.add_argument("--replicas-per-cta", type=int, default=0)
    p.add_argument("--threads", type=int, default=0)
    p.add_argument("--variant", type=int, default=2,
                   help="0 int8/int16 fields, 1 multi-spin coded, 2 automatic (default), 3 CTA pairs")
    p.add_argument("--hex", action="store_true")
    p.add_argument("--save-hex", default=None)
    p.add_argument("--curve", default=None, help="write step,beta,t_ms,best_cut CSV")
    p.add_argument("--checkpoint", default=None, help="checkpoint file written during the run")
    p.add_argument("--checkpoint-every", type=int, default=0, help="steps between checkpoints")
    p.add_argument("--resume", default=None, help="continue the anneal saved in this checkpoint")
    p.add_argument("--adaptive", type=int, default=0,
                   help="0 fixed schedule, 1 ESS-adaptive steps, 2 acceptance-rate-adaptive steps")
    p.add_argument("--rho", type=float, default=0.5, help="adaptive 1: target ESS / R")
    p.add_argument("--adapt-J", type=int, default=8, help="adaptive: finest grid level")
    p.add_argument("--dbeta-max", type=float, default=0.05, help="adaptive: coarsest step")
    p.add_argument("--beta-max", type=float, default=None, help="adaptive: final beta (default: the schedule's end)")
    p.add_argument("--acc-lo", type=float, default=0.05, help="adaptive 2: lower acceptance bound")
    p.add_argument("--acc-hi", type=float, default=0.25, help="adaptive 2: upper acceptance bound")
    p.add_argument("--reheat-after", type=int, default=0, help="fixed schedules: stagnant steps before a reheat")
    p.add_argument("--reheat-back", type=int, default=1, help="schedule entries a reheat steps back")
    a = p.parse_args(argv)
    build_mod.build()
    if a.graph:
        g = wl.read_gset(a.graph)
        c = dict(DEFAULT_FILE_SCHEDULE)
        name = a.graph
    else:
        name = a.config or "g63like"
        c = dict(wl.CONFIGS[name])
        g = c["graph"]()
    if a.beta is not None:
        c["beta"], c["K"] = (a.beta[0], a.beta[1]), int(a.beta[2])
    for key, val in (("R", a.replicas), ("S", a.sweeps), ("nlm_period", a.nlm_period), ("seed", a.seed)):
        if val is not None:
            c[key] = val
    betas = wl.linear_betas(*c["beta"], c["K"])
    K = c["K"] if a.steps is None else min(a.steps, c["K"])
    with B.Annealer.from_graph(g) as ann:
        t0 = time.perf_counter()
        if a.resume:
            ann.load(a.resume)
            c["R"], c["S"] = ann.R, ann.S
            K = ann.K if a.steps is None else min(a.steps, ann.K)
            done = B.pa_run_info(ann.ctx)["steps_done"]
        else:
            ctl = dict(reheat_after=a.reheat_after, reheat_back=a.reheat_back)
            if a.adaptive:
                ctl = dict(adaptive=a.adaptive, rho=a.rho, adapt_J=a.adapt_J, adapt_dbeta_max=a.dbeta_max,
                           beta_max=a.beta_max if a.beta_max is not None else c["beta"][1],
                           acc_lo=a.acc_lo, acc_hi=a.acc_hi)
            ann.begin(None if a.adaptive else betas, c["R"], c["S"], c["seed"], K=c["K"],
                      nlm_period=c["nlm_period"], field_bits=a.field_bits, replicas_per_cta=a.replicas_per_cta,
                      threads_per_cta=a.threads, variant=a.variant, nlm_kind=a.nlm_kind, nlm_block=a.nlm_block,
                      **ctl)
            done = 0
        every = a.checkpoint_every if a.checkpoint and a.checkpoint_every > 0 else max(K - done, 1)
        while done < K:
            done = min(K, done + every)
            ann.run(done)
            if a.checkpoint:
                ann.save(a.checkpoint)   # waits for the enqueued steps
        ann.sync()
        dt = time.perf_counter() - t0
        st = ann.stats()
        cut, cfg, step, sweep = ann.best()
        ss_all = ann.step_stats()
        ss_nlm = (ss_all["nlm_pairs"].sum(), ss_all["nlm_flips"].sum())
        if a.curve:
            ss = ann.step_stats()
            W = st["total_weight"]
            best = np.minimum.accumulate(ss["sweep_emin"].min(axis=1)) if len(ss["beta"]) else []
            with open(a.curve, "w") as f:
                f.write("step,beta,t_ms,best_cut\n")
                for k in range(len(ss["beta"])):
                    f.write(f"{k},{ss['beta'][k]:.17g},{ss['t_ms'][k]:.3f},{(W - int(best[k])) // 2}\n")
    out = dict(config=name, n=g.n, m=g.m, R=c["R"], S=c["S"], steps=int(st["steps_run"]), seed=c["seed"],
               best_cut=cut,
               best_step=step, best_sweep=sweep, wall_s=dt, attempts=st["attempts"],
               nlm_moves=int(ss_nlm[0]), nlm_flips=int(ss_nlm[1]),
               accepts=st["accepts"], device_ms=st["anneal_ms"], time_to_best_ms=st["t_best_ms"],
               attempts_per_s=st["attempts"] / max(st["anneal_ms"], 1e-9) * 1e3)
    if a.hex or a.save_hex:
        h = hexconfig.encode(cfg)
        if a.hex:
            out["config_hex"] = h
        if a.save_hex:
            with open(a.save_hex, "w") as f:
                f.write(h + "\n")
    print(json.dumps(out))
    return 0


def main(argv=None):
    argv = sys.argv[1:] if argv is None else list(argv)
    if argv and argv[0] == "verify":
        return _verify(argv[1:])
    return _anneal(argv)


if __name__ == "__main__":
    sys.exit(main())
