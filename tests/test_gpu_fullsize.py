"""Parity at the full benchmark sizes, in the launch configuration the
benchmark times: the GPU runs the real workload up to step k, its population
is dumped, and the oracle replays step k (resampling from the full energy
vector, then the sweeps and non-local moves of sampled slots) for comparison
with the GPU's population after step k."""
import numpy as np
import pytest

import oracle
from gpu_helpers import require_gpu
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _replay_check(g, betas, R, S, seed, k, subset, nlm_period=0, nlm_block=0, **opts):
    a = B.Annealer.from_graph(g)
    if nlm_block:
        opts.update(nlm_kind=1, nlm_block=nlm_block)
    a.begin(betas, R, S, seed, record_counts=1, nlm_period=nlm_period, **opts)
    a.run(k)
    a.sync()
    spins_a, E_a = a.state()
    a.run(k + 1)
    a.sync()
    spins_b, E_b = a.state()
    counts = a.step_stats(counts=True)["counts"][k]
    a.close()
    nlm_now = nlm_period > 0 and k > 0 and k % nlm_period == 0
    rep = oracle.step_replay(g.rp, g.col, g.w, spins_a, S, seed, k, betas[k - 1] if k else 0.0,
                             betas[k], subset, nlm_now=nlm_now, nlm_block=nlm_block)
    np.testing.assert_array_equal(counts, rep["counts"], err_msg="copy counts at full size")
    assert counts.sum() == R
    np.testing.assert_array_equal(spins_b[subset], rep["spins"], err_msg="replayed spins")
    np.testing.assert_array_equal(E_b[subset], rep["E"], err_msg="replayed energies")
    for s in subset[:4]:   # energies carried by the GPU equal a full recomputation
        assert oracle.energy(g.rp, g.col, g.w, spins_b[s]) == E_b[s]
    return E_a


@pytest.mark.parametrize("field_bits,variant", [(0, 2), (16, 0), (0, 1), (0, 3)])
def test_replay_g63like_full_population(field_bits, variant):
    c = wl.CONFIGS["g63like"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    subset = np.array([0, 1, 2, 3, 4097, 8190, 12345, 16383])
    _replay_check(g, betas, c["R"], c["S"], c["seed"], 3, subset, field_bits=field_bits, variant=variant)


def test_replay_g63like_nonlocal_step():
    c = wl.CONFIGS["g63like"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    k = c["nlm_period"]
    order = oracle.nlm_order(c["R"], c["seed"], k)
    subset = np.array(sorted(order[[0, 1, 2000, 2001, 16382, 16383]].tolist()))
    _replay_check(g, betas, c["R"], c["S"], c["seed"], k, subset, nlm_period=k)


def test_replay_g63like_block_move_step():
    """Block moves (b = 32) at the first non-local step of the full workload,
    in the launch configuration of the benchmark (multi-spin-coded sweeps)."""
    c = wl.CONFIGS["g63like"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    k = c["nlm_period"]
    subset = np.array([0, 1, 2, 3, 777, 4096, 9999, 16383])
    _replay_check(g, betas, c["R"], c["S"], c["seed"], k, subset, nlm_period=k, nlm_block=32)


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_replay_torus100_full_population(variant):
    c = wl.CONFIGS["torus100"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    subset = np.array([0, 5, 31, 32767, 20000])
    _replay_check(g, betas, c["R"], c["S"], c["seed"], 4, subset, variant=variant)


def test_replay_g63like_late_beta_default_layout():
    """Step 899 (beta = 3.61) of the benchmarked anneal in its own launch
    configuration: default layout (456 words in one-CTA blocks + 56 in CTA
    pairs), Houdayer moves every 50 steps before it. Low acceptance: most
    thresholds of the step's table are 0 ("never")."""
    c = wl.CONFIGS["g63like"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    k = 899
    T = oracle.accept_table(betas[k], g.maxdeg)
    assert (T[4:] == 0).all() and T[1] > 0
    subset = np.array([0, 1, 2, 3, 31, 4097, 8190, 12345, 14591, 14592, 15000, 16383])
    _replay_check(g, betas, c["R"], c["S"], c["seed"], k, subset, nlm_period=c["nlm_period"])


def test_replay_g63like_late_nonlocal_step():
    """Step 900 (beta = 3.61), a non-local step late in the benchmarked anneal,
    default layout: resampling, sweeps and Houdayer moves of sampled pairs."""
    c = wl.CONFIGS["g63like"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    k = 900
    assert k % c["nlm_period"] == 0
    order = oracle.nlm_order(c["R"], c["seed"], k)
    subset = np.array(sorted(order[[0, 1, 5000, 5001, 9998, 9999, 16382, 16383]].tolist()))
    _replay_check(g, betas, c["R"], c["S"], c["seed"], k, subset, nlm_period=c["nlm_period"])


@pytest.mark.parametrize("variant", [1, 3])
def test_replay_torus100_late_beta(variant):
    """Step 700 (beta = 3.08) of the 100 x 100 signed torus at R = 32768 in the
    multi-spin-coded kernels (one-CTA head + CTA-pair tail, and CTA pairs
    only)."""
    c = wl.CONFIGS["torus100"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    subset = np.array([0, 5, 31, 32, 9999, 20000, 29183, 29184, 32767])
    _replay_check(g, betas, c["R"], c["S"], c["seed"], 700, subset, variant=variant)


def test_full_g63like_anneal_properties():
    """The whole benchmarked anneal: invariants that hold at any size."""
    c = wl.CONFIGS["g63like"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    a = B.Annealer.from_graph(g)
    a.anneal(betas, c["R"], c["S"], c["seed"], nlm_period=c["nlm_period"])
    cut, cfg, step, sweep = a.best()
    Eb, sb, swb, slot = a.best_record()
    st = a.stats()
    rec = a.step_stats()
    a.close()
    W = oracle.total_weight(g.rp, g.col, g.w)
    assert oracle.energy(g.rp, g.col, g.w, cfg) == Eb and cut == (W - Eb) // 2
    assert Eb == rec["sweep_emin"].min()
    assert st["steps_run"] == c["K"] and st["attempts"] == g.n * c["R"] * c["S"] * c["K"]
    assert np.all(rec["nlm_pairs"][c["nlm_period"]::c["nlm_period"]] > 0)
    assert np.all(rec["T"] > 0)
    # a G63-shaped random graph: the cut should be far above the random-cut value M/2
    assert cut > 0.62 * g.m


def test_replay_maximum_replica_count():
    """R = 65536, the largest population the ABI takes: 2048 words, 1976 in
    one-CTA blocks and 72 in CTA pairs; copy counts of all slots and the
    spins of sampled slots replayed by the oracle at step 2."""
    c = wl.CONFIGS["g63like"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    subset = np.array([0, 31, 32, 4096, 63231, 63232, 65535])
    _replay_check(g, betas, 65536, 2, c["seed"], 2, subset)
