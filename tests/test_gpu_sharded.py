"""The device side of replica sharding (pa_shard_min, pa_shard_partials,
pa_shard_parents, pa_shard_gather) on one GPU: the population entering a step
of a real anneal is split into G = 1, 2, 4, 8 aligned slot ranges, each range
goes through the shard kernels, the host plan (pa_shard_plan) combines them,
and the copy counts, A (bitwise), T, E_min and the resampled rows must equal
the resampling inside pa_anneal (the library's single-population path) and the
oracle's. The collectives themselves are covered on CPU ranks
(test_sharded_cpu.py); this box has one GPU."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import require_gpu
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import sharded
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 7])
def test_shard_kernels_equal_single_population_resampling(k):
    require_gpu()
    import torch

    g = wl.gnm(3000, 18000, seed=5)
    betas = wl.linear_betas(0.2, 3.0, 12)
    R, S, seed = 4096, 2, 11
    a = B.Annealer.from_graph(g)
    a.begin(betas, R, S, seed, record_counts=1)
    a.run(k)
    a.sync()
    spins_in, E_in = a.state()          # population entering step k
    a.run(k + 1)
    a.sync()
    rec = a.step_stats(counts=True)
    a.close()
    o = sharded.resample_offset(seed, k)
    assert o == int(rec["o"][k])
    ref = oracle.resample(E_in, math.exp(-(betas[k] - betas[k - 1])), o)
    np.testing.assert_array_equal(ref["counts"], rec["counts"][k])
    dev = torch.device("cuda:0")
    for G in (1, 2, 4, 8):
        shards = [sharded.shard_range(R, G, h) for h in range(G)]
        locs = [sharded.LibraryShard(hi - lo, dev) for lo, hi in shards]
        Es = [torch.from_numpy(E_in[lo:hi].copy()).to(dev) for lo, hi in shards]
        Ss = [torch.from_numpy(spins_in[lo:hi].copy()).to(dev) for lo, hi in shards]
        emin = min(loc.emin(E) for loc, E in zip(locs, Es))
        parts = [loc.partials(E, emin, betas[k - 1], betas[k]) for loc, E in zip(locs, Es)]
        A_all = [p[0] for p in parts]
        T_all = [p[1] for p in parts]
        new_spins, new_E, counts = [], [], []
        for h, loc in enumerate(locs):
            p = sharded.plan(G, h, R, A_all, T_all, o)
            assert np.float64(p["A"]).view(np.uint64) == rec["A"][k:k + 1].view(np.uint64)[0], f"A, G={G}"
            assert p["T"] == int(rec["T"][k]) and emin == int(rec["emin"][k])
            src, c = loc.parents(R, o, p)
            rows, erows = loc.gather(Ss[h], Es[h], src)
            new_spins.append(rows.cpu().numpy())
            new_E.append(erows.cpu().numpy())
            counts.append(c.cpu().numpy())
        np.testing.assert_array_equal(np.concatenate(counts), rec["counts"][k], err_msg=f"counts, G={G}")
        np.testing.assert_array_equal(np.concatenate(new_spins), spins_in[ref["parent"]], err_msg=f"rows, G={G}")
        np.testing.assert_array_equal(np.concatenate(new_E), E_in[ref["parent"]], err_msg=f"energies, G={G}")
