"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
binding and the oracle on the same seeded inputs and compare."""
import numpy as np
import pytest

import oracle
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import build as build_mod


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build_mod.build()
    B.lib()


def run_gpu(g, betas, R, S, seed, K=None, counts=True, **opts):
    a = B.Annealer.from_graph(g)
    a.anneal(betas, R, S, seed, K=K, record_counts=int(counts), **opts)
    spins, E = a.state()
    rec = a.step_stats(counts=counts)
    best = a.best_record() if rec["beta"].size and S > 0 else None
    cut, cfg, _, _ = a.best() if best is not None else (None, None, None, None)
    stats = a.stats()
    a.close()
    return dict(spins=spins, E=E, rec=rec, best=best, cut=cut, cfg=cfg, stats=stats)


def run_oracle(g, betas, R, S, seed, K=None, counts=True, **opts):
    return oracle.anneal(g.rp, g.col, g.w, betas, R=R, S=S, seed=seed, K=K, record_counts=counts,
                         **opts)


def assert_parity(gpu, orc, g, R, S):
    steps = orc.steps_run
    assert gpu["stats"]["steps_run"] == steps
    rec = gpu["rec"]
    np.testing.assert_array_equal(rec["emin"], orc.step_emin, err_msg="E_min per step")
    assert np.array_equal(rec["A"].view(np.uint64), orc.step_A.view(np.uint64)), "weight sums A (bitwise)"
    np.testing.assert_array_equal(rec["T"], orc.step_T, err_msg="integer weight totals")
    np.testing.assert_array_equal(rec["o"], orc.step_o, err_msg="resampling offsets")
    np.testing.assert_array_equal(rec["beta"], orc.step_beta, err_msg="beta per step")
    if rec.get("counts") is not None and orc.step_counts is not None:
        np.testing.assert_array_equal(rec["counts"], orc.step_counts, err_msg="copy counts")
    np.testing.assert_array_equal(rec["accepts"], orc.step_accepts, err_msg="accepted flips")
    if S > 0:
        np.testing.assert_array_equal(rec["sweep_emin"], orc.step_sweep_emin, err_msg="sweep minima")
    np.testing.assert_array_equal(rec["nlm_pairs"], orc.step_nlm_pairs, err_msg="non-local pairs")
    np.testing.assert_array_equal(rec["nlm_flips"], orc.step_nlm_flips, err_msg="non-local flips")
    np.testing.assert_allclose(rec["lnZ"], orc.step_lnZ, rtol=1e-12, atol=1e-9)
    np.testing.assert_array_equal(gpu["E"], orc.E, err_msg="final energies")
    np.testing.assert_array_equal(gpu["spins"], orc.spins, err_msg="final spins")
    if S > 0 and steps > 0:
        assert gpu["best"] == (orc.best_E, orc.best_step, orc.best_sweep, orc.best_slot)
        np.testing.assert_array_equal(gpu["cfg"], orc.best_config, err_msg="best configuration")
        W = oracle.total_weight(g.rp, g.col, g.w)
        assert gpu["cut"] == (W - orc.best_E) // 2
        assert oracle.energy(g.rp, g.col, g.w, gpu["cfg"]) == orc.best_E
    assert gpu["stats"]["accepts"] == int(orc.step_accepts.sum())
    assert gpu["stats"]["attempts"] == g.n * R * S * steps
