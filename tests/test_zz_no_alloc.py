"""pa_resample_noalloc: the allocation-free resampling entry point, for callers
that cannot allocate device memory (stream capture into CUDA graphs, device
budgets owned by a host framework, loops that forbid allocator calls).

Its copy counts, parents, weight sum, integer total, minimum and offset must
equal those of the resampling inside pa_anneal (the existing entry point) on
the same energies, bit for bit, on two calls in a row. This file is named to
be collected last."""
import numpy as np
import pytest

from gpu_helpers import require_gpu
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_resample_matches_anneal_two_calls_in_a_row():
    require_gpu()
    import torch

    g = wl.gnm(3000, 18000, seed=5)
    betas = wl.linear_betas(0.2, 3.0, 10)
    R, S, seed = 4096, 2, 11
    a = B.Annealer.from_graph(g)
    a.begin(betas, R, S, seed, record_counts=1)
    _, E0 = a.state()            # energies entering step 0
    a.run(1)
    a.sync()
    _, E1 = a.state()            # energies entering step 1
    a.run(2)
    a.sync()
    rec = a.step_stats(counts=True)
    a.close()

    dev = torch.device("cuda:0")
    parent = torch.empty(R, dtype=torch.int32, device=dev)
    counts = torch.empty(R, dtype=torch.int32, device=dev)
    stream = B.current_stream_handle()
    for k, (E, bprev) in enumerate([(E0, 0.0), (E1, betas[0])]):
        Ed = torch.from_numpy(E).to(dev)
        res = B.pa_resample_noalloc(Ed.data_ptr(), R, bprev, betas[k], seed, k, parent.data_ptr(),
                                    counts.data_ptr(), stream)
        torch.cuda.synchronize()
        c = counts.cpu().numpy()
        np.testing.assert_array_equal(c, rec["counts"][k], err_msg=f"copy counts, call {k + 1}")
        np.testing.assert_array_equal(parent.cpu().numpy(), np.repeat(np.arange(R, dtype=np.int32), c))
        assert np.float64(res["A"]).view(np.uint64) == rec["A"][k:k + 1].view(np.uint64)[0]
        assert res["T"] == int(rec["T"][k]) and res["emin"] == int(rec["emin"][k])
        assert res["o"] == int(rec["o"][k])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    require_gpu()
    import torch

    R = 32769
    E = torch.zeros(R, dtype=torch.int32, device="cuda:0")
    parent = torch.empty(R, dtype=torch.int32, device="cuda:0")
    with pytest.raises(B.PaError) as e:
        B.pa_resample_noalloc(E.data_ptr(), R, 0.0, 1.0, 1, 0, parent.data_ptr())
    assert e.value.code == B.PA_EINVAL
