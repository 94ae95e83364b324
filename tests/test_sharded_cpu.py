"""Replica sharding of the resampling step on CPU ranks (gloo, world sizes 2
and 4): the plan and exchange of paper_2510_21105_gb300.sharded (pa_shard_plan
on the host, three collectives), with each rank's local arithmetic done by the
oracle, against the single-process oracle resampling of the whole population:
E_min, A (bitwise), T, every copy count and the resampled population (spins
and energies, slot by slot), over several steps whose weight concentrates on
a few replicas (many copies cross rank boundaries)."""
import math
import socket

import numpy as np
import pytest

import oracle
from paper_2510_21105_gb300 import sharded
from paper_2510_21105_gb300 import workloads as wl


class OracleShard:
    """A rank's local arithmetic by the oracle (stand-in for the library's
    kernels on ranks without a GPU)."""

    def __init__(self, n):
        self.n = n

    def emin(self, E):
        return int(E.min().item())

    def partials(self, E, emin, beta_prev, beta_k):
        A, T, t = oracle.shard_partials(E.numpy(), emin, math.exp(-(beta_k - beta_prev)))
        self.t = [int(x) for x in t]
        self.pre = [0] * self.n
        acc = 0
        for r in range(self.n):
            self.pre[r] = acc
            acc += self.t[r]
        return A, T

    def parents(self, R, o, step):
        import torch

        src = np.zeros(step["new_hi"] - step["new_lo"], np.int32)
        counts = np.zeros(self.n, np.int32)
        for r in range(self.n):
            P = step["P_base"] + self.pre[r]
            lo = oracle.systematic_count(P, R, step["T"], o)
            hi = oracle.systematic_count(P + self.t[r], R, step["T"], o)
            src[lo - step["new_lo"]:hi - step["new_lo"]] = r
            counts[r] = hi - lo
        return torch.from_numpy(src), torch.from_numpy(counts)

    def gather(self, spins, E, src):
        idx = src.long()
        return spins[idx].contiguous(), E[idx].contiguous()


STEPS = [(0.0, 0.3), (0.3, 0.9), (0.9, 2.5), (2.5, 6.0)]


def _population(R, seed=7):
    g = wl.gnm(40, 120, seed=3)
    rng = np.random.Generator(np.random.PCG64(seed))
    spins = np.where(rng.random((R, g.n)) < 0.5, 1, -1).astype(np.int8)
    E = np.array([oracle.energy(g.rp, g.col, g.w, x) for x in spins], np.int32)
    return spins, E


def _worker(rank, world, port, R, seed):
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        full_spins, full_E = _population(R)
        lo, hi = sharded.shard_range(R, world, rank)
        res = sharded.ShardedResampler(R, OracleShard(hi - lo), dist)
        spins = torch.from_numpy(full_spins[lo:hi].copy())
        E = torch.from_numpy(full_E[lo:hi].copy())
        crossed = 0
        for k, (bp, bk) in enumerate(STEPS):
            spins, E, rec = res.step(spins, E, bp, bk, seed, k)
            o = sharded.resample_offset(seed, k)
            ref = oracle.resample(full_E, math.exp(-(bk - bp)), o)
            assert rec["o"] == int(oracle.philox4x32_10([0, 0, k, 1 << 28], [seed & 0xFFFFFFFF, seed >> 32])[0])
            assert rec["emin"] == ref["emin"] and rec["T"] == ref["T"]
            assert np.float64(rec["A"]).view(np.uint64) == np.float64(ref["A"]).view(np.uint64), "A (bitwise)"
            counts = [torch.zeros(hi - lo, dtype=torch.int32) for _ in range(world)]
            dist.all_gather(counts, rec["counts"].to(torch.int32))
            np.testing.assert_array_equal(torch.cat(counts).numpy(), ref["counts"], err_msg=f"counts, step {k}")
            full_spins = full_spins[ref["parent"]]
            full_E = full_E[ref["parent"]]
            np.testing.assert_array_equal(spins.numpy(), full_spins[lo:hi], err_msg=f"spins, step {k}")
            np.testing.assert_array_equal(E.numpy(), full_E[lo:hi], err_msg=f"energies, step {k}")
            crossed += int(np.sum((ref["parent"][lo:hi] < lo) | (ref["parent"][lo:hi] >= hi)))
        assert crossed > 0   # rows did move between ranks
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_resampling_equals_single_population(world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    torch.set_num_threads(1)
    mp.spawn(_worker, args=(world, _free_port(), 256, 0x5EED_1234_ABCD), nprocs=world, join=True)


def test_plan_is_the_single_population_tree_top_and_partition():
    """pa_shard_plan alone (host): the new-slot ranges of the ranks tile
    [0, R) in rank order, send and receive counts agree across ranks, and A is
    the pairwise tree over the rank sums."""
    R, G = 1024, 8
    rng = np.random.Generator(np.random.PCG64(11))
    A_all = list(rng.random(G) * 50)
    T_all = [int(x) for x in rng.integers(1, 2**40, G)]
    o = 0x9ABCDEF1
    plans = [sharded.plan(G, g, R, A_all, T_all, o) for g in range(G)]
    lvl = list(A_all)
    while len(lvl) > 1:
        lvl = [lvl[2 * i] + lvl[2 * i + 1] for i in range(len(lvl) // 2)]
    assert all(np.float64(p["A"]).view(np.uint64) == np.float64(lvl[0]).view(np.uint64) for p in plans)
    assert plans[0]["new_lo"] == 0 and plans[-1]["new_hi"] == R
    for a, b in zip(plans, plans[1:]):
        assert a["new_hi"] == b["new_lo"]
    for g in range(G):
        for h in range(G):
            assert plans[g]["send"][h] == plans[h]["recv"][g]
        assert sum(plans[g]["recv"]) == R // G
        assert sum(plans[g]["send"]) == plans[g]["new_hi"] - plans[g]["new_lo"]
