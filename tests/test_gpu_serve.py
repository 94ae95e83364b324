"""Serving loop (pa_server_*): requests admitted by device-memory budget while
others run produce results bit-identical to the same requests run alone, and
each request run alone is bit-identical to the oracle."""
import time

import numpy as np
import pytest

from gpu_helpers import assert_parity, require_gpu, run_gpu, run_oracle
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _requests():
    return [
        (wl.gnm(2000, 12000, seed=11), wl.linear_betas(0.1, 3.0, 30), 256, 4, 1, dict()),
        (wl.torus(40, seed=12), wl.linear_betas(0.1, 3.5, 25), 512, 3, 2, dict(variant=1)),
        (wl.gnp(400, 0.05, seed=13), wl.linear_betas(0.2, 2.5, 40), 96, 2, 3, dict(nlm_period=10)),
        (wl.delaunay(3000, seed=14), wl.linear_betas(0.1, 3.0, 20), 1024, 2, 4, dict(field_bits=16)),
        (wl.gnm(1200, 6000, seed=15), wl.linear_betas(0.1, 2.0, 15), 64, 5, 5, dict()),
        (wl.torus(30, seed=16), wl.linear_betas(0.1, 3.0, 35), 200, 2, 6, dict()),
    ]


def test_each_request_alone_matches_oracle():
    """Every request of the served mix, run alone, against the oracle element by
    element (spins, energies, per-step records, copy counts, best record)."""
    require_gpu()
    for g, betas, R, S, seed, kw in _requests():
        gpu = run_gpu(g, betas, R, S, seed, **kw)
        orc = run_oracle(g, betas, R, S, seed, **{k: v for k, v in kw.items() if k == "nlm_period"})
        assert_parity(gpu, orc, g, R, S)


def _alone(g, betas, R, S, seed, kw):
    with B.Annealer.from_graph(g) as a:
        a.anneal(betas, R, S, seed, **kw)
        cut, cfg, _, _ = a.best()
        return a.best_record(), cut, cfg


@pytest.mark.parametrize("budget_mb,streams,tick", [(8192, 4, 4), (40, 2, 3)])
def test_served_results_equal_alone(budget_mb, streams, tick):
    require_gpu()
    reqs = _requests()
    ref = [_alone(*r) for r in reqs]
    with B.Server(budget_mb << 20, n_streams=streams, steps_per_tick=tick) as srv:
        ids = []
        for i, (g, betas, R, S, seed, kw) in enumerate(reqs):
            ids.append(srv.submit(g, betas, R, S, seed, **kw))
            if i % 2 == 1:
                time.sleep(0.02)   # later requests arrive while earlier ones run
            st = srv.stats()
            assert st["bytes_in_use"] <= (budget_mb << 20) or st["running"] <= 1
        done = {}
        t_end = time.time() + 120
        while len(done) < len(ids) and time.time() < t_end:
            for rid in ids:
                if rid not in done and srv.poll(rid) == 2:
                    done[rid] = srv.result(rid)
            time.sleep(0.005)
        assert len(done) == len(ids)
        for rid, (best, cut, cfg) in zip(ids, ref):
            r = done[rid]
            assert r["status"] == 0
            assert (r["energy"], r["step"], r["sweep"], r["slot"]) == best
            assert r["cut"] == cut and np.array_equal(r["config"], cfg)
            assert r["finish_ms"] >= r["start_ms"] >= r["submit_ms"]
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["queued"] == 0 and st["running"] == 0


def test_server_rejects_bad_requests():
    require_gpu()
    with B.Server(1 << 30) as srv:
        g = wl.gnp(50, 0.1, seed=1)
        with pytest.raises(B.PaError):
            srv.submit(g, None, 8, 2, 0, K=5)     # K steps but no schedule, and not adaptive
        rid = srv.submit(g, [0.5, 0.4], 8, 2, 0)  # decreasing schedule: fails at admission
        t_end = time.time() + 30
        while srv.poll(rid) in (0, 1) and time.time() < t_end:
            time.sleep(0.005)
        assert srv.poll(rid) == B.PA_EINVAL
