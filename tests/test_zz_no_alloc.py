"""pa_resample_noalloc: the resampling entry point that allocates no device
memory, for callers that cannot call cudaMalloc (a host framework that owns
the device-memory budget through its own pool, loops where an allocator call
may block or synchronise the device).

Its copy counts, parents, weight sum, integer total, minimum and offset must
equal, bit for bit and on two calls in a row:
  - those of the resampling inside pa_anneal (the existing entry point) on
    the energies of a real anneal;
  - those of the oracle's resampling (Sec. 3, systematic resampling with
    fixed R) on the same energies, for populations that are not powers of
    two (the zero-padded pairwise tree), a single replica, and the largest
    population its fixed scratch takes (PA_NOALLOC_MAX_R = 32768).
This file is named to be collected last."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import require_gpu
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MAX_R = 32768


def _offset_word(seed: int, k: int) -> int:
    """Word 0 of Philox(0, 0, k, tag 1) keyed by the seed (the offset o)."""
    return int(oracle.philox4x32_10([0, 0, k, 1 << 28], [seed & 0xFFFFFFFF, seed >> 32])[0])


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


@pytest.mark.parametrize("R", [1, 3000, 4955, MAX_R])
def test_noalloc_resample_matches_oracle(R):
    """Two calls in a row on energies of different spread (one with weights
    that underflow to zero), each against the oracle's resampling."""
    require_gpu()
    import torch

    rng = np.random.Generator(np.random.PCG64(1000 + R))
    dev = torch.device("cuda:0")
    parent = torch.full((R,), -1, dtype=torch.int32, device=dev)
    counts = torch.full((R,), -1, dtype=torch.int32, device=dev)
    stream = B.current_stream_handle()
    seed = 0x1234_5678_9ABC + R
    calls = [
        # late-anneal shape: E near a minimum, beta step of a 1000-step schedule
        (-27000 + rng.geometric(0.02, R).astype(np.int32) * 2, 3.5, 3.5039, 901),
        # wide spread and a large beta step: most weights underflow
        (rng.integers(-41000, 41000, R, dtype=np.int32), 0.1, 0.6, 3),
    ]
    for i, (E, bprev, bk, k) in enumerate(calls):
        E = np.ascontiguousarray(E, dtype=np.int32)
        Ed = torch.from_numpy(E).to(dev)
        res = B.pa_resample_noalloc(Ed.data_ptr(), R, bprev, bk, seed, k, parent.data_ptr(),
                                    counts.data_ptr(), stream)
        torch.cuda.synchronize()
        ref = oracle.resample(E, math.exp(-(bk - bprev)), _offset_word(seed, k))
        np.testing.assert_array_equal(counts.cpu().numpy(), ref["counts"], err_msg=f"copy counts, call {i + 1}")
        np.testing.assert_array_equal(parent.cpu().numpy(), ref["parent"], err_msg=f"parents, call {i + 1}")
        assert np.float64(res["A"]).view(np.uint64) == np.float64(ref["A"]).view(np.uint64), "A (bitwise)"
        assert res["T"] == ref["T"] and res["emin"] == ref["emin"]
        assert res["o"] == _offset_word(seed, k)
        assert int(ref["counts"].sum()) == R


def test_noalloc_without_host_result():
    """With no host result requested (NULL) the call only enqueues its kernel;
    the copy counts are the same as with the result."""
    require_gpu()
    import torch

    R, seed, k = 3000, 77, 5
    E = np.random.Generator(np.random.PCG64(3)).integers(-9000, -8000, R, dtype=np.int32)
    dev = torch.device("cuda:0")
    Ed = torch.from_numpy(E).to(dev)
    parent = torch.empty(R, dtype=torch.int32, device=dev)
    counts = torch.empty(R, dtype=torch.int32, device=dev)
    stream = B.current_stream_handle()
    out = B.pa_resample_noalloc(Ed.data_ptr(), R, 1.0, 1.01, seed, k, parent.data_ptr(), counts.data_ptr(),
                                stream, want_result=False)
    assert out is None
    torch.cuda.synchronize()
    ref = oracle.resample(E, math.exp(-(1.01 - 1.0)), _offset_word(seed, k))
    np.testing.assert_array_equal(counts.cpu().numpy(), ref["counts"])
    np.testing.assert_array_equal(parent.cpu().numpy(), ref["parent"])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    require_gpu()
    import torch

    R = MAX_R + 1
    E = torch.zeros(R, dtype=torch.int32, device="cuda:0")
    parent = torch.empty(R, dtype=torch.int32, device="cuda:0")
    with pytest.raises(B.PaError) as e:
        B.pa_resample_noalloc(E.data_ptr(), R, 0.0, 1.0, 1, 0, parent.data_ptr())
    assert e.value.code == B.PA_EINVAL
