"""Batched anneals (pa_batch_anneal): each job's results are bit-identical to the
same job run alone, with concurrent streams and with one captured CUDA graph;
each job run alone is bit-identical to the oracle."""
import numpy as np
import pytest

from gpu_helpers import assert_parity, require_gpu, run_gpu, run_oracle
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _jobs():
    return [
        (wl.gnp(300, 0.05, seed=1), wl.linear_betas(0.1, 2.5, 9), 16, 3, 5, dict()),
        (wl.torus(20, seed=2), wl.linear_betas(0.1, 3.0, 12), 40, 2, 6, dict(variant=1)),
        (wl.delaunay(500, seed=3), wl.linear_betas(0.2, 2.0, 7), 13, 4, 7, dict(field_bits=16)),
        (wl.gnm(1000, 5000, seed=4), wl.linear_betas(0.1, 3.0, 11), 64, 2, 8, dict(nlm_period=4)),
        (wl.gnm(800, 3000, seed=5), None, 32, 2, 9,
         dict(adaptive=1, rho=0.5, adapt_J=4, adapt_dbeta_max=0.3, beta_max=1.5)),
        (wl.gnp(150, 0.1, seed=6), wl.linear_betas(0.3, 1.0, 3), 7, 1, 10, dict(field_bits=8)),
        (wl.gnm(600, 3600, seed=7), wl.linear_betas(0.1, 2.5, 6), 5000, 2, 11, dict(variant=1, msc_no_split=1)),
    ]


ORACLE_KEYS = ("nlm_period", "adaptive", "rho", "adapt_J", "adapt_dbeta_max", "beta_max", "nlm_kind",
               "nlm_block", "acc_lo", "acc_hi", "reheat_after", "reheat_back")


def test_each_job_alone_matches_oracle():
    """Every job of the batch, run alone, against the oracle element by element
    (spins, energies, per-step records, copy counts, best record)."""
    require_gpu()
    for g, betas, R, S, seed, kw in _jobs():
        K = 60 if betas is None else None
        gpu = run_gpu(g, betas, R, S, seed, K=K, **kw)
        orc = run_oracle(g, betas, R, S, seed, K=K, **{k: v for k, v in kw.items() if k in ORACLE_KEYS})
        assert_parity(gpu, orc, g, R, S)


def _alone(g, betas, R, S, seed, kw):
    K = 60 if betas is None else len(betas)
    with B.Annealer.from_graph(g) as a:
        a.anneal(betas, R, S, seed, K=K, **kw)
        return a.state(), a.best_record(), a.step_stats()["accepts"]


@pytest.mark.parametrize("use_graph,n_streams", [(False, 3), (True, 4), (False, 1)])
def test_batch_equals_alone(use_graph, n_streams):
    require_gpu()
    jobs = _jobs()
    ref = [_alone(*j) for j in jobs]
    anns = [B.Annealer.from_graph(j[0]) for j in jobs]
    items = [(ann, betas, R, S, seed, 60 if betas is None else len(betas), kw)
             for ann, (g, betas, R, S, seed, kw) in zip(anns, jobs)]
    ms = B.pa_batch_anneal(items, n_streams=n_streams, use_graph=use_graph)
    assert ms > 0
    for ann, (state, best, acc) in zip(anns, ref):
        s, E = ann.state()
        assert np.array_equal(s, state[0]) and np.array_equal(E, state[1])
        assert ann.best_record() == best
        assert np.array_equal(ann.step_stats()["accepts"], acc)
        ann.close()
