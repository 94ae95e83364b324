"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test checks one oracle function against mathematics, a library routine,
brute force or a value the paper prints, so that a dropped term, a wrong sign
or index, or a transposed operand in the oracle fails here.
"""
import ctypes as C
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2510_21105_gb300 import hexconfig, workloads as wl


# ---------------------------------------------------------------- Philox ---
def _curand_host_sequence(seed: int, count: int):
    """cuRAND's host-side Philox4x32-10 generator (runs on the CPU)."""
    path = None
    for cand in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so"):
        try:
            lib = C.CDLL(cand)
            path = cand
            break
        except OSError:
            continue
    if path is None:
        pytest.skip("libcurand not available")
    gen = C.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(C.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
    out = np.zeros(count, np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(C.c_void_p), C.c_size_t(count)) == 0
    lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 0xFEDCBA9876543210])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host generator emits block b as Philox(counter = (b // 65536, 0, b % 65536, 0),
    # key = seed): this pins the key words and counter words 0 and 2.
    seq = _curand_host_sequence(seed, 4 * 65536 * 2).reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in [0, 1, 2, 77, 4095, 65535, 65536, 65536 + 12345, 2 * 65536 - 1]:
        ctr = [b // 65536, 0, b % 65536, 0]
        assert np.array_equal(oracle.philox4x32_10(ctr, key), seq[b]), b


def test_philox_matches_triton_reference_all_counter_words():
    # Triton's Philox4x32 (library source, run by its CPU interpreter) on counters
    # with all four words non-zero pins words 1 and 3 as well.
    pytest.importorskip("triton")
    code = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
from triton.language.random import philox
@triton.jit
def k(c_ptr, out_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = philox(seed, tl.load(c_ptr + i * 4), tl.load(c_ptr + i * 4 + 1),
                        tl.load(c_ptr + i * 4 + 2), tl.load(c_ptr + i * 4 + 3), 10)
    tl.store(out_ptr + i * 4, a); tl.store(out_ptr + i * 4 + 1, b)
    tl.store(out_ptr + i * 4 + 2, c); tl.store(out_ptr + i * 4 + 3, d)
rng = np.random.default_rng(5)
ctr = torch.from_numpy(rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).astype(np.uint32))
out = torch.zeros_like(ctr)
k[(1,)](ctr, out, int(sys.argv[1]), n=16)
np.save(sys.argv[2], np.concatenate([ctr.numpy(), out.numpy()], 1))
"""
    import tempfile
    seed = 0x9E3779B97F4A7C15
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "p.npy")
        try:
            subprocess.run([sys.executable, "-c", code, str(seed), f], check=True, timeout=600,
                           capture_output=True)
        except (subprocess.CalledProcessError, subprocess.TimeoutExpired) as e:
            pytest.skip(f"triton interpreter unavailable: {e}")
        arr = np.load(f)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for row in arr:
        assert np.array_equal(oracle.philox4x32_10(row[:4], key), row[4:])


# ------------------------------------------------------------- colouring ---
def test_greedy_colour_matches_networkx_first_fit():
    nx = pytest.importorskip("networkx")
    for g in [wl.gnp(120, 0.1, seed=3), wl.gnm(500, 2000, seed=4), wl.delaunay(300, seed=5)]:
        ncol, colour = oracle.greedy_colour(g.rp, g.col)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        i, j, _ = g.edges()
        G.add_edges_from(zip(i.tolist(), j.tolist()))
        ref = nx.greedy_color(G, strategy=lambda G, colors: range(G.number_of_nodes()))
        assert [ref[v] for v in range(g.n)] == colour.tolist()
        assert ncol == max(ref.values()) + 1
        # every colour class is an independent set
        assert not np.any(colour[i] == colour[j])


def test_even_torus_is_two_coloured_checkerboard():
    g = wl.torus(100, seed=0)
    ncol, colour = oracle.greedy_colour(g.rp, g.col)
    assert ncol == 2
    r, c = np.divmod(np.arange(g.n), 100)
    assert np.array_equal(colour, (r + c) % 2)


# ------------------------------------------------------------ energy/cut ---
def test_cut_identity_against_direct_edge_count():
    rng = np.random.default_rng(0)
    for g in [wl.gnp(200, 0.05, seed=1), wl.torus(12, seed=2)]:
        i, j, w = g.edges()
        W = oracle.total_weight(g.rp, g.col, g.w)
        assert W == int(w.sum())
        for _ in range(5):
            x = rng.choice(np.array([-1, 1], np.int8), size=g.n)
            E = oracle.energy(g.rp, g.col, g.w, x)
            cut = int(w[x[i] != x[j]].sum())          # Eq. 1 counted edge by edge
            assert (W - E) % 2 == 0
            assert (W - E) // 2 == cut


def _brute_force_maxcut(g):
    i, j, w = g.edges()
    n = g.n
    states = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int8)
    cut = ((states[:, i] != states[:, j]) * w[None, :]).sum(1)
    return int(cut.max())


def test_best_cut_reaches_brute_force_optimum_on_small_graphs():
    for seed, g in enumerate([wl.gnp(14, 0.4, seed=7), wl.torus(4, seed=8), wl.gnm(16, 40, seed=9)]):
        best = _brute_force_maxcut(g)
        W = oracle.total_weight(g.rp, g.col, g.w)
        res = oracle.anneal(g.rp, g.col, g.w, wl.linear_betas(0.1, 3.0, 30), R=64, S=4, seed=seed)
        cut = (W - res.best_E) // 2
        assert cut <= best
        assert cut == best
        assert oracle.energy(g.rp, g.col, g.w, res.best_config) == res.best_E


def test_final_energies_equal_full_recomputation():
    g = wl.gnp(150, 0.08, seed=11)
    res = oracle.anneal(g.rp, g.col, g.w, wl.linear_betas(0.2, 2.0, 12), R=40, S=3, seed=5,
                        nlm_period=4)
    for r in range(40):
        assert res.E[r] == oracle.energy(g.rp, g.col, g.w, res.spins[r])
    # best tracking: the best equals the minimum over every sweep end
    assert res.best_E == int(res.step_sweep_emin.min())
    k, s = np.unravel_index(np.argmin(res.step_sweep_emin), res.step_sweep_emin.shape)
    assert (res.best_step, res.best_sweep) == (k, s)


# -------------------------------------------------------------- Metropolis ---
def _exact_boltzmann(g, beta):
    i, j, w = g.edges()
    n = g.n
    states = np.where(((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1) == 1, 1, -1)
    E = (states[:, i] * states[:, j] * w[None, :]).sum(1)
    p = np.exp(-beta * (E - E.min()))
    return p / p.sum(), E


def test_fixed_beta_histogram_matches_boltzmann_chi_square():
    from scipy.stats import chisquare

    g = wl.from_edges(7, [0, 0, 1, 2, 3, 4, 5, 1, 2], [1, 2, 3, 4, 5, 6, 6, 5, 6],
                      [1, -1, 1, 1, -1, 1, 1, 1, -1])
    beta = 0.45
    p, _ = _exact_boltzmann(g, beta)
    nsamp = 6000
    counts = np.zeros(2 ** g.n)
    for seed in range(nsamp):
        res = oracle.anneal(g.rp, g.col, g.w, np.full(2, beta), R=1, S=12, seed=seed)
        idx = int(((res.spins[0] == 1).astype(np.int64) << np.arange(g.n)).sum())
        counts[idx] += 1
    expected = p * nsamp
    keep = expected >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(expected[keep], expected[~keep].sum())
    stat = chisquare(obs, exp)
    assert stat.pvalue > 1e-3, stat


def test_sweep_uniform_is_uniform_at_full_resolution():
    """The Metropolis uniform of an attempt takes its top byte from a Philox
    call shared by 16 replicas and its low 24 bits from a second stream. It
    must be uniform on [0, 2^32): P(u < T) = T / 2^32 also for thresholds
    inside one top-byte band, where a comparison of the top byte alone (or
    with a constant tail) is off by up to 1/256; replicas that share a call
    draw different top bytes."""
    from scipy.stats import chisquare

    n = 1 << 21
    verts = np.arange(n) % 7000          # distinct (vertex, replica) pairs
    slots = np.arange(n) // 7000
    u = oracle.sweep_uniforms(0x1234_5678_9ABC, verts, slots, 17, 3).astype(np.int64)
    assert chisquare(np.bincount(u >> 28, minlength=16)).pvalue > 1e-3
    sigma = math.sqrt(0.25 / n)
    for T in (0x80000001, 0x80800000, 0x80FFFFFF):
        assert abs(np.mean(u < T) - T / 2.0 ** 32) < 5 * sigma, hex(T)
    # the 16 replicas of one call, and the tail stream: pairwise independent top bytes
    v = np.arange(1 << 16)
    top = np.stack([oracle.sweep_uniforms(9, v, np.full(v.size, r), 4, 0) >> 24 for r in range(16)])
    for a, b in [(0, 1), (0, 4), (3, 15), (5, 6)]:
        assert abs(np.mean(top[a] == top[b]) - 1 / 256) < 5 * math.sqrt(1 / 256 / v.size)
    low = oracle.sweep_uniforms(9, v, np.full(v.size, 2), 4, 0) & 0xFFFFFF
    assert chisquare(np.bincount(low >> 20, minlength=16)).pvalue > 1e-3


def test_parallel_timing_build_equals_checking_build():
    """The OpenMP build (replicas swept on several threads, used only to time
    the oracle on all host cores) gives the single-thread results bit for bit."""
    g = wl.gnm(500, 3000, seed=3)
    betas = wl.linear_betas(0.1, 3.0, 12)
    a = oracle.anneal(g.rp, g.col, g.w, betas, R=48, S=3, seed=5, nlm_period=4, record_counts=True)
    oracle.lib_parallel(4)
    p = oracle.anneal(g.rp, g.col, g.w, betas, R=48, S=3, seed=5, nlm_period=4, record_counts=True, parallel=True)
    assert np.array_equal(a.spins, p.spins) and np.array_equal(a.E, p.E)
    assert np.array_equal(a.step_accepts, p.step_accepts) and np.array_equal(a.step_counts, p.step_counts)
    assert np.array_equal(a.step_A.view(np.uint64), p.step_A.view(np.uint64))
    assert (a.best_E, a.best_step, a.best_sweep, a.best_slot) == (p.best_E, p.best_step, p.best_sweep, p.best_slot)


def test_accept_table_is_floor_of_boltzmann_factor():
    for beta in [0.0, 0.1, 1.0, 3.7]:
        T = oracle.accept_table(beta, 40)
        assert T[0] == 0xFFFFFFFF
        assert np.all(np.diff(T[1:].astype(np.int64)) <= 0)
        for m in range(1, 41):
            ref = min(2.0 ** 32 - 1, math.floor(math.ldexp(math.exp(-beta * 2 * m), 32)))
            assert abs(int(T[m]) - ref) <= 1


# ------------------------------------------------------------- resampling ---
def test_resample_identity_at_zero_dbeta_and_count_sum():
    rng = np.random.default_rng(1)
    E = rng.integers(-300, 300, size=1000).astype(np.int32)
    out = oracle.resample(E, 1.0, 0x12345678)
    assert np.all(out["counts"] == 1)
    assert np.array_equal(out["parent"], np.arange(1000))
    for q in [0.99, 0.9, 0.5, 1e-3]:
        for o in [0, 1, 2**31, 2**32 - 1]:
            r = oracle.resample(E, q, o)
            assert r["counts"].sum() == 1000
            assert np.all(np.diff(r["parent"]) >= 0)
            assert np.array_equal(np.bincount(r["parent"], minlength=1000), r["counts"])


def test_resample_mean_copies_equal_normalised_weights():
    rng = np.random.default_rng(2)
    R = 64
    E = rng.integers(-40, 40, size=R).astype(np.int32)
    q = math.exp(-0.07)
    L = 4096
    mean = np.zeros(R)
    for t in range(L):
        o = (t * (2**32 // L)) + 12345
        mean += oracle.resample(E, q, o)["counts"]
    mean /= L
    w = q ** (E - E.min()).astype(np.float64)
    assert np.allclose(mean, R * w / w.sum(), atol=2.0 / L + 1e-6)
    r = oracle.resample(E, q, 7)
    assert r["emin"] == E.min()
    assert math.isclose(r["A"], w.sum(), rel_tol=1e-12)


def test_free_energy_estimate_matches_exact_partition_function():
    g = wl.gnp(10, 0.45, seed=21)
    beta_f = 1.2
    betas = wl.linear_betas(0.06, beta_f, 20)
    p, E = _exact_boltzmann(g, beta_f)
    lnZ_exact = math.log(np.exp(-beta_f * E.astype(np.float64)).sum())
    est = []
    for seed in range(24):
        res = oracle.anneal(g.rp, g.col, g.w, betas, R=2048, S=2, seed=seed)
        est.append(res.step_lnZ[-1])
    est = np.array(est)
    err = est.std(ddof=1) / math.sqrt(len(est))
    assert abs(est.mean() - lnZ_exact) < 4 * err + 0.01, (est.mean(), lnZ_exact, err)


# ------------------------------------------------------------ non-local ---
def test_houdayer_cluster_is_connected_component_and_conserves_energy():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(3)
    for g in [wl.gnp(80, 0.05, seed=31), wl.torus(8, seed=32)]:
        i, j, _ = g.edges()
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(zip(i.tolist(), j.tolist()))
        for trial in range(20):
            xa = rng.choice(np.array([-1, 1], np.int8), size=g.n)
            xb = xa.copy()
            flipmask = rng.random(g.n) < 0.4
            xb[flipmask] *= -1
            u = int(rng.integers(0, 2**32))
            size, ya, yb, cl = oracle.houdayer_pair(g.rp, g.col, xa, xb, u)
            D = np.flatnonzero(xa != xb)
            if len(D) == 0:
                assert size == 0
                continue
            seedv = int(D[u % len(D)])
            comp = nx.node_connected_component(G.subgraph(D.tolist()), seedv)
            assert set(np.flatnonzero(cl).tolist()) == comp
            assert size == len(comp)
            ea = oracle.energy(g.rp, g.col, g.w, xa) + oracle.energy(g.rp, g.col, g.w, xb)
            eb = oracle.energy(g.rp, g.col, g.w, ya) + oracle.energy(g.rp, g.col, g.w, yb)
            assert ea == eb
            # on the cluster the two replicas exchange their values
            assert np.array_equal(ya[cl], xb[cl]) and np.array_equal(yb[cl], xa[cl])
            assert np.array_equal(ya[~cl], xa[~cl]) and np.array_equal(yb[~cl], xb[~cl])


def _edge_energy(g, x):
    """E = sum over undirected edges of w x_i x_j, from the edge list."""
    i, j, w = g.edges()
    return int(np.sum(w.astype(np.int64) * x[i] * x[j]))


def test_block_move_block_is_bfs_prefix_and_energy_change_is_exact():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(5)
    for g in [wl.gnp(90, 0.06, seed=41), wl.torus(9, seed=42), wl.gnm(200, 500, seed=43)]:
        i, j, _ = g.edges()
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(zip(i.tolist(), j.tolist()))
        for trial in range(25):
            x = rng.choice(np.array([-1, 1], np.int8), size=g.n)
            E = _edge_energy(g, x)
            b = int(rng.integers(1, 40))
            sv = int(rng.integers(0, g.n))
            order = [sv] + [v for _, v in nx.bfs_edges(G, sv, sort_neighbors=sorted)]
            want = set(order[:b])
            size, y, E2, mask = oracle.block_move(g.rp, g.col, g.w, x, E, b, 1.0, sv, 0)
            assert set(np.flatnonzero(mask).tolist()) == want
            # q = 1 (beta = 0): every move is accepted
            assert size == len(want)
            flipped = x.copy()
            flipped[list(want)] *= -1
            assert np.array_equal(y, flipped)
            assert E2 == _edge_energy(g, flipped)


def test_block_move_acceptance_threshold_is_boltzmann_factor():
    mp = pytest.importorskip("mpmath")
    g = wl.gnm(120, 400, seed=44)
    rng = np.random.default_rng(6)
    checked = 0
    for trial in range(200):
        x = rng.choice(np.array([-1, 1], np.int8), size=g.n)
        E = _edge_energy(g, x)
        sv, b = int(rng.integers(0, g.n)), int(rng.integers(1, 12))
        _, y, E1, mask = oracle.block_move(g.rp, g.col, g.w, x, E, b, 1.0, sv, 0)
        m = (E1 - E) // 2
        beta = float(rng.uniform(0.05, 1.0))
        q = math.exp(-2.0 * beta)
        if m <= 0:
            size, *_ = oracle.block_move(g.rp, g.col, g.w, x, E, b, q, sv, 2**32 - 1)
            assert size == int(mask.sum())
            continue
        exact = int(mp.floor(mp.ldexp(mp.exp(-2 * mp.mpf(beta) * m), 32)))
        if exact < 4:
            continue
        acc_lo, *_ = oracle.block_move(g.rp, g.col, g.w, x, E, b, q, sv, exact - 2)
        acc_hi, *_ = oracle.block_move(g.rp, g.col, g.w, x, E, b, q, sv, exact + 1)
        assert acc_lo == int(mask.sum()) and acc_hi == 0
        checked += 1
    assert checked > 20


def test_block_move_of_one_spin_is_a_metropolis_flip():
    g = wl.gnp(60, 0.1, seed=45)
    rng = np.random.default_rng(7)
    beta = 0.7
    T = oracle.accept_table(beta, g.maxdeg)
    for trial in range(60):
        x = rng.choice(np.array([-1, 1], np.int8), size=g.n)
        E = _edge_energy(g, x)
        v = int(rng.integers(0, g.n))
        row = g.col[g.rp[v]:g.rp[v + 1]]
        m = int(-x[v] * x[row].sum())          # unweighted: h_v = sum of neighbour spins
        u = int(rng.integers(0, 2**32))
        size, y, E2, _ = oracle.block_move(g.rp, g.col, g.w, x, E, 1, math.exp(-2.0 * beta), v, u)
        if m <= 0:
            assert size == 1 and E2 == E + 2 * m
        elif abs(int(u) - int(T[m])) > 2:      # away from the rounding of the threshold
            assert (size == 1) == (u < int(T[m]))


def test_block_move_covers_whole_component_when_b_is_large():
    nx = pytest.importorskip("networkx")
    g = wl.from_edges(10, [0, 1, 2, 5, 6], [1, 2, 3, 6, 7])
    i, j, _ = g.edges()
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(zip(i.tolist(), j.tolist()))
    x = np.ones(g.n, np.int8)
    size, y, E2, mask = oracle.block_move(g.rp, g.col, g.w, x, _edge_energy(g, x), 100, 1.0, 2, 0)
    assert set(np.flatnonzero(mask).tolist()) == nx.node_connected_component(G, 2) == {0, 1, 2, 3}
    assert size == 4 and E2 == _edge_energy(g, y)


def test_nlm_pairing_is_a_permutation():
    order = oracle.nlm_order(1000, 42, 50)
    assert sorted(order.tolist()) == list(range(1000))
    assert not np.array_equal(order, np.arange(1000))


# ------------------------------------------------------------ adaptive ---
def test_adaptive_steps_meet_ess_threshold():
    g = wl.gnp(60, 0.1, seed=41)
    R, J, dmax, bmax, rho = 512, 6, 0.2, 2.0, 0.6
    res = oracle.anneal(g.rp, g.col, g.w, None, R=R, S=2, seed=3, K=400, adaptive=True,
                        rho=rho, adapt_J=J, adapt_dbeta_max=dmax, beta_max=bmax)
    delta = math.ldexp(dmax, -J)
    n = np.rint(res.step_beta / delta).astype(np.int64)
    assert np.allclose(n * delta, res.step_beta, rtol=0, atol=1e-12)
    dn = np.diff(np.concatenate([[0], n]))
    assert np.all(dn >= 1)
    assert res.step_beta[-1] == pytest.approx(bmax)
    nmax = int(math.floor(bmax / delta + 0.5))
    for k in range(res.steps_run):
        if n[k] < nmax:   # unclamped step: dn is the power of two of the chosen level
            assert dn[k] == 2 ** (J - res.step_jsel[k])
    # First step, checked independently from the initial population (K = 0 run).
    init = oracle.anneal(g.rp, g.col, g.w, np.zeros(0), R=R, S=2, seed=3)
    E0 = init.E.astype(np.float64)
    j_expected = J
    for j in range(J + 1):
        w = np.exp(-(2 ** (J - j)) * delta * (E0 - E0.min()))
        if w.sum() ** 2 / (w * w).sum() >= rho * R:
            j_expected = j
            break
    assert res.step_jsel[0] == j_expected


# ------------------------------------------------------------ step replay ---
def test_step_replay_reproduces_full_run():
    g = wl.gnp(90, 0.07, seed=51)
    betas = wl.linear_betas(0.1, 2.5, 10)
    R, S, seed, k = 48, 3, 9, 6
    before = oracle.anneal(g.rp, g.col, g.w, betas[:k], R=R, S=S, seed=seed)
    after = oracle.anneal(g.rp, g.col, g.w, betas[:k + 1], R=R, S=S, seed=seed, record_counts=True)
    sub = np.array([0, 5, 17, 47])
    rep = oracle.step_replay(g.rp, g.col, g.w, before.spins, S, seed, k, betas[k - 1], betas[k], sub)
    assert np.array_equal(rep["spins"], after.spins[sub])
    assert np.array_equal(rep["E"], after.E[sub])
    assert np.array_equal(rep["counts"], after.step_counts[k])


# ------------------------------------------------------------ paper format ---
def test_paper_configuration_decodes_to_7000_spins(golden_dir):
    lines = open(os.path.join(golden_dir, "g63_best_config.txt")).read().splitlines()
    hexstr = "".join(l.strip() for l in lines if l and not l.startswith("#"))
    assert len(hexstr) == 1750
    x = hexconfig.decode(hexstr, 7000)
    assert len(x) == 7000
    assert int((x == 1).sum()) == 3425 and int((x == -1).sum()) == 3575
    assert x[0] == 1 and x[1] == 1 and x[2] == -1     # leading digit 'd' = 1101
    assert hexconfig.encode(x) == hexstr


def test_hex_roundtrip_odd_lengths():
    rng = np.random.default_rng(0)
    for n in [1, 3, 4, 5, 17, 801]:
        x = rng.choice(np.array([-1, 1], np.int8), size=n)
        assert np.array_equal(hexconfig.decode(hexconfig.encode(x), n), x)


def test_anneal_with_block_moves_keeps_energies_exact():
    """Whole anneals with block moves: carried energies equal recomputation,
    every move is counted, and b = 1 moves flip one spin each."""
    g = wl.torus(10, seed=46)
    betas = wl.linear_betas(0.02, 0.3, 12)     # hot enough for blocks of 40 to be accepted
    for b in (1, 7, 40):
        res = oracle.anneal(g.rp, g.col, g.w, betas, R=24, S=1, seed=9, nlm_period=3, nlm_kind=1, nlm_block=b)
        for r in range(24):
            assert res.E[r] == _edge_energy(g, res.spins[r])
        due = [k for k in range(12) if k > 0 and k % 3 == 0]
        assert np.all(res.step_nlm_pairs[[k for k in range(12) if k not in due]] == 0)
        assert res.step_nlm_pairs[due].sum() > 0
        assert np.all(res.step_nlm_flips <= b * res.step_nlm_pairs)
        if b == 1:
            assert np.array_equal(res.step_nlm_flips, res.step_nlm_pairs)


def test_acceptance_rate_control_follows_recorded_rates():
    """adaptive = 2: the level sequence recomputed from the recorded accepted
    flips (which the sweeps pins above fix), and beta advances by the grid
    step of each level, monotonically, to beta_max."""
    g = wl.gnm(150, 600, seed=47)
    R, S, J, dmax, bmax, lo, hi = 40, 2, 4, 0.4, 3.0, 0.12, 0.3
    res = oracle.anneal(g.rp, g.col, g.w, None, R=R, S=S, seed=3, K=400, adaptive=2, adapt_J=J,
                        adapt_dbeta_max=dmax, beta_max=bmax, acc_lo=lo, acc_hi=hi)
    K = res.steps_run
    assert 0 < K < 400
    delta = math.ldexp(dmax, -J)
    nmax = int(math.floor(bmax / delta + 0.5))
    attempts = g.n * R * S
    j, n_prev = 0, 0
    seen = set()
    for k in range(K):
        if k > 0:
            rate = res.step_accepts[k - 1]
            if rate < lo * attempts:
                j = min(j + 1, J)
            elif rate > hi * attempts:
                j = max(j - 1, 0)
        seen.add(j)
        assert res.step_jsel[k] == j
        n_prev += min(2 ** (J - j), nmax - n_prev)
        assert res.step_beta[k] == n_prev * delta
    assert res.step_beta[-1] == pytest.approx(bmax)
    assert len(seen) >= 3                      # the band moves the level both ways
    assert np.all(np.diff(res.step_beta) > 0)


def test_stagnation_reheating_follows_recorded_minima():
    """reheat_after > 0: the schedule index sequence recomputed from the
    recorded sweep minima; steps that do not advance the index resample with
    q = 1, which is the identity (every copy count 1, A = R)."""
    g = wl.gnm(150, 600, seed=47)
    betas = wl.linear_betas(0.1, 3.0, 60)
    R, S, Q, back = 32, 2, 3, 10
    res = oracle.anneal(g.rp, g.col, g.w, betas, R=R, S=S, seed=4, reheat_after=Q, reheat_back=back,
                        record_counts=True)
    i_prev, stall, best = 0, 0, 2**31 - 1
    reheats = 0
    for k in range(60):
        i = 0
        if k > 0:
            m = int(res.step_sweep_emin[k - 1].min())
            if m < best:
                best, stall = m, 0
            else:
                stall += 1
            if stall >= Q:
                i, stall = max(0, i_prev - back), 0
                reheats += 1
            else:
                i = min(i_prev + 1, 59)
        assert res.step_jsel[k] == i
        assert res.step_beta[k] == betas[i]
        if k > 0 and i != i_prev + 1:
            assert np.all(res.step_counts[k] == 1) and res.step_A[k] == R
        i_prev = i
    assert reheats >= 2
    plain = oracle.anneal(g.rp, g.col, g.w, betas, R=R, S=S, seed=4)
    assert not np.array_equal(plain.step_beta, res.step_beta)
