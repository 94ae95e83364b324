"""GPU path vs oracle, element by element, through the C-ABI (bit-exact:
spins, energies, copy counts, weight sums, best record and configuration)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_parity, require_gpu, run_gpu, run_oracle
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_tables_and_colouring_match_oracle():
    g = wl.gnp(300, 0.07, seed=3)
    betas = wl.linear_betas(0.1, 3.0, 9)
    a = B.Annealer.from_graph(g)
    a.begin(betas, R=8, S=1, seed=1)
    for k in range(9):
        acc, _ = a.tables(k, g.maxdeg)
        assert np.array_equal(acc, oracle.accept_table(betas[k], g.maxdeg))
    ncol, colour, pos = a.colouring()
    ncol_o, colour_o = oracle.greedy_colour(g.rp, g.col)
    assert ncol == ncol_o and np.array_equal(colour, colour_o)
    assert sorted(pos.tolist()) == list(range(g.n))
    a.close()


@pytest.mark.parametrize("field_bits,variant", [(0, 0), (16, 0), (0, 1), (0, 3)])
def test_parity_gnp800_full_workload(field_bits, variant):
    # N = 800, p = 0.06, R = 256, beta 0.1 -> 3.0 in 100 steps, 4 sweeps, seed 0.
    c = wl.CONFIGS["gnp800"]
    g = c["graph"]()
    betas = wl.linear_betas(*c["beta"], c["K"])
    gpu = run_gpu(g, betas, c["R"], c["S"], c["seed"], field_bits=field_bits, variant=variant)
    orc = _oracle_cached("gnp800", lambda: run_oracle(g, betas, c["R"], c["S"], c["seed"]))
    assert_parity(gpu, orc, g, c["R"], c["S"])


_ORACLE_CACHE = {}


def _oracle_cached(key, fn):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = fn()
    return _ORACLE_CACHE[key]


@pytest.mark.parametrize("R,opts", [(6, {}), (6, {"field_bits": 16}), (13, {"field_bits": 8}),
                                    (1, {}), (1, {"field_bits": 16}), (7, {"field_bits": 7, "threads_per_cta": 256}),
                                    (24, {"replicas_per_cta": 8, "field_bits": 16}),
                                    (40, {"replicas_per_cta": 8, "field_bits": 8, "threads_per_cta": 128}),
                                    (6, {"variant": 1}), (33, {"variant": 1}), (70, {"variant": 1, "threads_per_cta": 128}),
                                    (1, {"variant": 3}), (40, {"variant": 3}), (97, {"variant": 3})])
def test_parity_ragged_signed(R, opts):
    g = wl.from_edges(37, *_random_edges(37, 90, seed=R), name="ragged")
    betas = wl.linear_betas(0.05, 2.5, 7)
    gpu = run_gpu(g, betas, R, 3, seed=1234 + R, **opts)
    orc = run_oracle(g, betas, R, 3, seed=1234 + R)
    assert_parity(gpu, orc, g, R, 3)


def _random_edges(n, m, seed):
    rng = np.random.default_rng(seed)
    seen = set()
    while len(seen) < m:
        i, j = sorted(rng.integers(0, n, 2).tolist())
        if i != j:
            seen.add((i, j))
    e = np.array(sorted(seen))
    w = rng.choice(np.array([-1, 1], np.int8), size=len(e))
    return e[:, 0], e[:, 1], w


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_parity_torus_two_colour_checkerboard(variant):
    g = wl.torus(24, seed=5)
    betas = wl.linear_betas(0.1, 3.5, 12)
    gpu = run_gpu(g, betas, 64, 4, seed=9, variant=variant)
    orc = run_oracle(g, betas, 64, 4, seed=9)
    assert gpu["stats"]["n_colours"] == 2
    assert_parity(gpu, orc, g, 64, 4)


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_parity_nonlocal_moves(variant):
    g = wl.gnm(500, 3000, seed=7)
    betas = wl.linear_betas(0.1, 3.0, 13)
    gpu = run_gpu(g, betas, 64, 3, seed=11, nlm_period=3, variant=variant)
    orc = run_oracle(g, betas, 64, 3, seed=11, nlm_period=3)
    assert orc.step_nlm_pairs.sum() > 0
    assert_parity(gpu, orc, g, 64, 3)


@pytest.mark.parametrize("R", [2, 8, 32, 33, 65])
def test_parity_nonlocal_moves_small_populations(R):
    """Houdayer pairing through key buckets at the smallest populations: one
    bucket (R <= 32), two and four buckets, and an odd R whose last slot stays
    unpaired."""
    g = wl.gnm(200, 800, seed=R)
    betas = wl.linear_betas(0.1, 2.5, 8)
    gpu = run_gpu(g, betas, R, 2, seed=5 + R, nlm_period=2)
    orc = run_oracle(g, betas, R, 2, seed=5 + R, nlm_period=2)
    assert orc.step_nlm_pairs.sum() > 0
    assert_parity(gpu, orc, g, R, 2)


@pytest.mark.parametrize("variant", [0, 1, 3])
@pytest.mark.parametrize("n,m", [(600, 900), (300, 3000)])
def test_parity_nonlocal_moves_low_and_high_degree(variant, n, m):
    """Houdayer moves on graphs of mean degree 3 (rows shorter than the group
    of 4 lanes that reads one) and 20 (five passes per row)."""
    g = wl.gnm(n, m, seed=n + m)
    betas = wl.linear_betas(0.1, 3.0, 9)
    gpu = run_gpu(g, betas, 128, 2, seed=17, nlm_period=2, variant=variant)
    orc = run_oracle(g, betas, 128, 2, seed=17, nlm_period=2)
    assert orc.step_nlm_pairs.sum() > 0 and orc.step_nlm_flips.sum() > 0
    assert_parity(gpu, orc, g, 128, 2)


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_parity_nonlocal_moves_signed(variant):
    """Houdayer moves on a +-1 torus: the multi-spin-coded layouts update the
    two energies from the bonds across the cluster boundary, the others
    recompute fields and energies; both must give the oracle's energies."""
    g = wl.torus(16, seed=21)
    betas = wl.linear_betas(0.2, 2.5, 10)
    gpu = run_gpu(g, betas, 96, 2, seed=4, nlm_period=2, variant=variant)
    orc = run_oracle(g, betas, 96, 2, seed=4, nlm_period=2)
    assert orc.step_nlm_pairs.sum() > 0 and orc.step_nlm_flips.sum() > 0
    assert_parity(gpu, orc, g, 96, 2)


@pytest.mark.parametrize("block", [1, 13, 300])
@pytest.mark.parametrize("variant,field_bits", [(0, 16), (0, 7), (1, 0), (3, 0)],
                         ids=["int16", "packed", "msc", "msc-pair"])
def test_parity_block_moves(variant, field_bits, block):
    """Block moves (nlm_kind = 1) on a signed graph in every layout: b = 1 is
    a single Metropolis flip, b = 300 covers the seed's whole component."""
    g = wl.from_edges(300, *_random_edges(300, 900, seed=55))
    betas = wl.linear_betas(0.02, 1.2, 10)
    kw = dict(nlm_period=2, nlm_kind=1, nlm_block=block)
    gpu = run_gpu(g, betas, 50, 2, seed=23, variant=variant, field_bits=field_bits, **kw)
    orc = run_oracle(g, betas, 50, 2, seed=23, **kw)
    assert orc.step_nlm_pairs.sum() > 0
    assert_parity(gpu, orc, g, 50, 2)


def test_parity_block_moves_adaptive():
    g = wl.gnp(150, 0.06, seed=56)
    kw = dict(adaptive=1, rho=0.6, adapt_J=4, adapt_dbeta_max=0.2, beta_max=1.0, nlm_period=2, nlm_kind=1,
              nlm_block=9)
    gpu = run_gpu(g, None, 64, 2, seed=29, K=200, **kw)
    orc = run_oracle(g, None, 64, 2, seed=29, K=200, **{**kw, "adaptive": True})
    assert orc.step_nlm_pairs.sum() > 0
    np.testing.assert_array_equal(gpu["rec"]["jsel"], orc.step_jsel)
    assert_parity(gpu, orc, g, 64, 2)


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_parity_acceptance_rate_control(variant):
    """adaptive = 2 (acceptance-rate rule), alone and with block moves."""
    g = wl.from_edges(250, *_random_edges(250, 1000, seed=58))
    kw = dict(adaptive=2, adapt_J=4, adapt_dbeta_max=0.4, beta_max=3.0, acc_lo=0.12, acc_hi=0.3)
    for extra in (dict(), dict(nlm_period=1, nlm_kind=1, nlm_block=2)):
        gpu = run_gpu(g, None, 72, 2, seed=37, K=400, variant=variant, **kw, **extra)
        orc = run_oracle(g, None, 72, 2, seed=37, K=400, **kw, **extra)
        assert 0 < orc.steps_run < 400 and len(set(orc.step_jsel.tolist())) >= 3
        np.testing.assert_array_equal(gpu["rec"]["jsel"], orc.step_jsel)
        assert_parity(gpu, orc, g, 72, 2)


@pytest.mark.parametrize("variant,field_bits", [(0, 16), (0, 7), (1, 0), (3, 0)],
                         ids=["int16", "packed", "msc", "msc-pair"])
def test_parity_stagnation_reheating(variant, field_bits):
    """Stagnation reheating on a fixed schedule, alone and with block moves;
    the schedule index of every step is compared."""
    g = wl.gnm(150, 600, seed=47)
    betas = wl.linear_betas(0.1, 3.0, 60)
    for extra in (dict(), dict(nlm_period=4, nlm_kind=1, nlm_block=3)):
        kw = dict(reheat_after=3, reheat_back=10, **extra)
        gpu = run_gpu(g, betas, 40, 2, seed=4, variant=variant, field_bits=field_bits, **kw)
        orc = run_oracle(g, betas, 40, 2, seed=4, **kw)
        assert len(set(np.diff(orc.step_jsel).tolist())) >= 2      # at least one reheat
        np.testing.assert_array_equal(gpu["rec"]["jsel"], orc.step_jsel)
        assert_parity(gpu, orc, g, 40, 2)


def test_block_move_options_are_validated():
    g = wl.gnp(50, 0.1, seed=57)
    a = B.Annealer.from_graph(g)
    for kw in (dict(nlm_kind=2), dict(nlm_kind=1, nlm_block=0), dict(nlm_kind=1, nlm_block=1025),
               dict(adaptive=3), dict(adaptive=2, acc_lo=0.5, acc_hi=0.4), dict(adaptive=2, acc_hi=1.5),
               dict(reheat_after=-1), dict(reheat_after=2, reheat_back=0),
               dict(reheat_after=2, reheat_back=1, adaptive=1, beta_max=1.0)):
        with pytest.raises(B.PaError) as e:
            a.begin(wl.linear_betas(0.1, 1.0, 3), R=8, S=1, seed=1, nlm_period=1, **kw)
        assert e.value.code == B.PA_EINVAL
    a.close()


def test_parity_adaptive_steps():
    g = wl.gnp(120, 0.08, seed=13)
    kw = dict(adaptive=1, rho=0.6, adapt_J=5, adapt_dbeta_max=0.25, beta_max=2.0)
    gpu = run_gpu(g, None, 96, 2, seed=17, K=300, **kw)
    orc = run_oracle(g, None, 96, 2, seed=17, K=300, adaptive=True, rho=0.6, adapt_J=5,
                     adapt_dbeta_max=0.25, beta_max=2.0)
    assert orc.steps_run < 300 and orc.step_beta[-1] == pytest.approx(2.0)
    np.testing.assert_array_equal(gpu["rec"]["jsel"], orc.step_jsel)
    assert_parity(gpu, orc, g, 96, 2)


def test_degenerate_cases():
    # Empty graph: every flip has dE = 0 and is accepted.
    g = wl.from_edges(5, [], [])
    betas = wl.linear_betas(0.5, 1.0, 3)
    gpu = run_gpu(g, betas, 4, 2, seed=3)
    orc = run_oracle(g, betas, 4, 2, seed=3)
    assert_parity(gpu, orc, g, 4, 2)
    # Zero sweeps: resampling only; no best exists.
    g = wl.gnp(30, 0.2, seed=1)
    a = B.Annealer.from_graph(g)
    a.anneal(wl.linear_betas(0.1, 1.0, 4), R=8, S=0, seed=2)
    with pytest.raises(B.PaError) as e:
        a.best()
    assert e.value.code == B.PA_ESTATE
    a.close()
    # Invalid schedules and sizes.
    a = B.Annealer.from_graph(g)
    for betas, R in [([0.5, 0.4], 8), ([0.1, np.nan], 8), ([0.1], 0), ([0.1], 70000), ([-0.1], 8)]:
        with pytest.raises(B.PaError) as e:
            a.anneal(np.array(betas), R=R, S=1, seed=0)
        assert e.value.code == B.PA_EINVAL
    a.close()


@pytest.mark.parametrize("variant,field_bits", [(0, 16), (0, 8), (0, 7), (1, 0), (3, 0)],
                         ids=["int16", "int8", "packed", "msc", "msc-pair"])
def test_degenerate_cases_every_layout(variant, field_bits):
    """Degenerate inputs in every layout, element by element against the oracle:
    a single vertex, an edgeless graph (every attempt has m = 0 and is accepted),
    one replica (plain simulated annealing: resampling is the identity), a
    single temperature step, and beta = 0 throughout (uniform acceptance)."""
    kw = dict(variant=variant, field_bits=field_bits)
    cases = [
        (wl.from_edges(1, [], []), wl.linear_betas(0.5, 1.0, 3), 5, 2),
        (wl.from_edges(50, [], []), wl.linear_betas(0.5, 1.0, 3), 33, 2),
        (wl.gnp(60, 0.1, seed=71), wl.linear_betas(0.1, 2.0, 6), 1, 3),
        (wl.torus(6, seed=72), np.array([0.7]), 40, 4),
        (wl.gnp(60, 0.1, seed=73), np.zeros(4), 36, 2),
    ]
    for g, betas, R, S in cases:
        gpu = run_gpu(g, betas, R, S, seed=5, **kw)
        orc = run_oracle(g, betas, R, S, seed=5)
        assert_parity(gpu, orc, g, R, S)
        if R == 1:
            assert np.all(orc.step_counts == 1)


@pytest.mark.parametrize("kw,K,split", [
    (dict(nlm_period=4), 10, 6),
    (dict(variant=1), 10, 3),
    (dict(variant=3, nlm_period=3), 10, 4),
    (dict(adaptive=1, rho=0.5, adapt_J=4, adapt_dbeta_max=0.3, beta_max=1.5, nlm_period=3), 40, 7),
    (dict(reheat_after=2, reheat_back=3, nlm_period=2, nlm_kind=1, nlm_block=4), 24, 11),
], ids=["fixed-nlm", "msc", "msc-pair", "adaptive", "reheat-block"])
def test_checkpoint_resume_is_bit_exact(tmp_path, kw, K, split):
    """A run saved after `split` steps and resumed in a fresh context equals
    the uninterrupted run: population, best record and every per-step record
    (the adaptive controller's state travels in the checkpoint)."""
    require_gpu()
    g = wl.gnp(200, 0.05, seed=21)
    betas = None if kw.get("adaptive") else wl.linear_betas(0.1, 2.5, K)
    full = B.Annealer.from_graph(g)
    full.anneal(betas, R=64, S=3, seed=5, K=K, **kw)
    s_full, E_full = full.state()
    b_full = full.best_record()
    st_full = full.step_stats()
    part = B.Annealer.from_graph(g)
    part.begin(betas, R=64, S=3, seed=5, K=K, **kw)
    part.run(split)
    part.sync()
    part.save(str(tmp_path / "ck.bin"))
    part.close()
    res = B.Annealer.from_graph(g)
    res.load(str(tmp_path / "ck.bin"))
    res.run(K)
    res.sync()
    s_res, E_res = res.state()
    assert np.array_equal(s_full, s_res) and np.array_equal(E_full, E_res)
    assert res.best_record() == b_full
    st_res = res.step_stats()
    assert len(st_res["beta"]) == len(st_full["beta"]) > split
    for key in ("beta", "emin", "A", "T", "o", "accepts", "sweep_emin", "nlm_pairs", "nlm_flips", "jsel", "lnZ"):
        assert np.array_equal(st_full[key], st_res[key]), key
    assert np.all(np.diff(st_res["t_ms"]) >= 0) and st_res["t_ms"][-1] > 0
    full.close()
    res.close()


def test_repeat_runs_are_identical_and_launch_shape_free():
    g = wl.gnm(1000, 6000, seed=3)
    betas = wl.linear_betas(0.2, 3.0, 6)
    r1 = run_gpu(g, betas, 64, 3, seed=77)
    r2 = run_gpu(g, betas, 64, 3, seed=77, threads_per_cta=256)
    r3 = run_gpu(g, betas, 64, 3, seed=77, replicas_per_cta=8, threads_per_cta=1024, field_bits=16)
    r4 = run_gpu(g, betas, 64, 3, seed=77, field_bits=8)
    r5 = run_gpu(g, betas, 64, 3, seed=77, field_bits=16)
    r6 = run_gpu(g, betas, 64, 3, seed=77, variant=1)
    for r in (r2, r3, r4, r5, r6):
        assert np.array_equal(r1["spins"], r["spins"]) and r1["best"] == r["best"]


@pytest.mark.parametrize("variant,extra", [(1, {}), (1, {"msc_no_split": 1}), (3, {})])
def test_parity_msc_many_words_ragged_last_word(variant, extra):
    # R = 4937: 155 words of 32 replicas (more words than SMs, so blocks loop
    # over words) with 9 live replicas in the last one; signed weights and
    # non-local moves. On 152 SMs the one-CTA layout splits the words 152 + 3
    # over two kernels unless msc_no_split asks for one.
    g = wl.from_edges(300, *_random_edges(300, 1500, seed=99))
    betas = wl.linear_betas(0.1, 2.5, 6)
    gpu = run_gpu(g, betas, 4937, 2, seed=31, variant=variant, nlm_period=2, **extra)
    orc = run_oracle(g, betas, 4937, 2, seed=31, nlm_period=2)
    assert_parity(gpu, orc, g, 4937, 2)


@pytest.mark.parametrize("variant", [1, 3])
def test_parity_msc_above_padded_rows(variant):
    """n = 17000 (> 16384 positions, beyond the 16-bit padded rows): the
    multi-spin-coded kernels read the plain CSR, with a single-bond tail per
    row; signed weights, mean degree 12, max degree above 15."""
    g = wl.from_edges(17000, *_random_edges(17000, 102000, seed=5))
    betas = wl.linear_betas(0.1, 2.5, 4)
    gpu = run_gpu(g, betas, 64, 2, seed=21, variant=variant)
    orc = run_oracle(g, betas, 64, 2, seed=21)
    assert_parity(gpu, orc, g, 64, 2)


def test_parity_largest_graph_that_fits_shared_memory():
    """n = 40000: too large for the packed (n <= 32720) and int16 layouts, so
    AUTO falls back to multi-spin coding even with fewer words than SMs; block
    moves and Houdayer moves (bitsets of both replicas and the candidates, a
    16-bit queue: 95 KB of shared memory per pair) both run at this size."""
    g = wl.gnm(40000, 60000, seed=61)
    betas = wl.linear_betas(0.2, 1.5, 3)
    gpu = run_gpu(g, betas, 40, 1, seed=3, nlm_period=2, nlm_kind=1, nlm_block=8)
    assert gpu["stats"]["variant"] == 1
    orc = run_oracle(g, betas, 40, 1, seed=3, nlm_period=2, nlm_kind=1, nlm_block=8)
    assert_parity(gpu, orc, g, 40, 1)
    gpu = run_gpu(g, betas, 40, 1, seed=3, nlm_period=2)
    assert gpu["stats"]["variant"] == 1
    orc = run_oracle(g, betas, 40, 1, seed=3, nlm_period=2)
    assert_parity(gpu, orc, g, 40, 1)


def test_layouts_that_do_not_fit_are_refused():
    """Graphs whose replica block exceeds the per-CTA shared memory are
    rejected with PA_EINVAL, not launched."""
    require_gpu()
    big = wl.gnm(60000, 60000, seed=62)       # 240 KB per multi-spin-coded block
    a = B.Annealer.from_graph(big)
    with pytest.raises(B.PaError) as e:
        a.begin(wl.linear_betas(0.2, 1.5, 2), R=64, S=1, seed=1)
    assert e.value.code == B.PA_EINVAL and "shared memory" in str(e.value)
    a.close()
    mid = wl.gnm(20000, 40000, seed=63)       # int16 layout: 240 KB; packed fits
    a = B.Annealer.from_graph(mid)
    with pytest.raises(B.PaError) as e:
        a.begin(wl.linear_betas(0.2, 1.5, 2), R=64, S=1, seed=1, field_bits=16)
    assert e.value.code == B.PA_EINVAL
    a.begin(wl.linear_betas(0.2, 1.5, 2), R=64, S=1, seed=1)
    a.run(2)
    a.sync()
    a.close()


@pytest.mark.parametrize("R,expect", [(1903, 0), (2500, 3), (4832, 3), (4865, 1)])
def test_auto_layout_choice_by_population(R, expect):
    """The default layout follows the number of 32-replica words against the
    SM count: packed below 40% of the SMs, the CTA-pair kernel up to one word
    per SM, then the one-CTA kernel (with its CTA-pair tail). Every choice
    gives the oracle's results."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    words = (R + 31) // 32
    want = 1 if words >= sms else (3 if 5 * words >= 2 * sms else 0)
    if sms == 152:
        assert want == expect
    g = wl.gnp(120, 0.1, seed=71)
    betas = wl.linear_betas(0.3, 2.0, 3)
    gpu = run_gpu(g, betas, R, 1, seed=5)
    assert gpu["stats"]["variant"] == want
    orc = run_oracle(g, betas, R, 1, seed=5)
    assert_parity(gpu, orc, g, R, 1)
