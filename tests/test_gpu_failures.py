"""Failure handling, with every failure made on the host (no kernel is made to
fault, trap or wait):

- a device allocator that fails the n-th allocation: every entry point that
  allocates reports PA_ENOMEM, and destroying the context returns every
  allocation it made (no leak); the next context works normally;
- a served request larger than the device-memory budget waits while another
  request runs (its result reads PA_EBUSY), then runs once memory frees;
- a served request whose host-side job stalls (the tick thread holds it) is
  cancelled with PA_ETIMEOUT after its timeout while the other requests
  complete with results identical to their lone runs."""
import time

import numpy as np
import pytest

from gpu_helpers import require_gpu
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


class _FailingAllocator:
    """torch-backed allocator that counts live allocations and returns NULL on
    the allocation with index fail_at (counted from the last reset)."""

    def __init__(self):
        import torch

        self.torch = torch
        self.live = {}
        self.count = 0
        self.fail_at = -1
        self.errors = []
        self.fns = (B.ALLOC_FN(self._alloc), B.FREE_FN(self._free))

    def _alloc(self, nbytes, _user):
        i = self.count
        self.count += 1
        if i == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes))
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, _user):
        if ptr not in self.live:
            self.errors.append(ptr)
            return
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)

    def reset(self, fail_at=-1):
        self.count = 0
        self.fail_at = fail_at


def _run(g, betas):
    a = B.Annealer.from_graph(g)
    try:
        a.anneal(betas, 64, 2, 5, nlm_period=2, record_counts=1)
        return a.state(), a.best_record()
    finally:
        a.close()


def test_allocation_failure_reports_enomem_and_leaks_nothing():
    require_gpu()
    import torch

    g = wl.gnm(300, 1500, seed=3)
    betas = wl.linear_betas(0.1, 2.0, 4)
    al = _FailingAllocator()
    B.lib().pa_set_allocator(al.fns[0], al.fns[1], None)
    try:
        al.reset()
        ref = _run(g, betas)
        total = al.count
        assert total >= 10 and not al.live
        for fail_at in range(total):
            al.reset(fail_at)
            with pytest.raises(B.PaError) as e:
                _run(g, betas)
            assert e.value.code == B.PA_ENOMEM, (fail_at, e.value)
            torch.cuda.synchronize()
            assert not al.live, f"allocation {fail_at} failed: {len(al.live)} allocations leaked"
        al.reset()
        again = _run(g, betas)
        assert np.array_equal(again[0][0], ref[0][0]) and np.array_equal(again[0][1], ref[0][1])
        assert again[1] == ref[1]
        assert not al.live and not al.errors
    finally:
        B.lib().pa_set_allocator(B.ALLOC_FN(0), B.FREE_FN(0), None)


def _alone_best(g, betas, R, S, seed):
    with B.Annealer.from_graph(g) as a:
        a.anneal(betas, R, S, seed)
        return a.best_record()


def _wait(srv, ids, timeout_s=120):
    t_end = time.time() + timeout_s
    while time.time() < t_end:
        if all(srv.poll(r) not in (0, 1) for r in ids):
            return True
        time.sleep(0.005)
    return False


def test_oversized_request_waits_for_memory():
    """Budget below the second request's footprint: it stays queued while the
    first runs (held on the host, so the check does not race the device), its
    result reads PA_EBUSY, and it runs once the first has finished and
    released its memory (a lone request is always admitted)."""
    require_gpu()
    g1, b1 = wl.gnm(2000, 12000, seed=21), wl.linear_betas(0.1, 3.0, 60)
    g2, b2 = wl.gnm(1500, 9000, seed=22), wl.linear_betas(0.1, 2.0, 10)
    with B.Server(64 << 20, n_streams=4, steps_per_tick=2) as srv:
        r1 = srv.submit(g1, b1, 2048, 4, 1)
        srv.hold(r1)
        t_end = time.time() + 30
        while srv.poll(r1) == 0 and time.time() < t_end:
            time.sleep(0.001)
        assert srv.poll(r1) == 1
        r2 = srv.submit(g2, b2, 8192, 2, 2)   # estimated footprint above the 64 MB budget
        time.sleep(0.2)
        assert srv.poll(r2) == 0 and srv.poll(r1) == 1
        assert srv.result(r2) is None                 # PA_EBUSY: not finished
        assert srv.release(r2) is False               # PA_EBUSY as well
        st = srv.stats()
        assert st["queued"] == 1 and st["running"] == 1
        srv.hold(r1, False)
        assert _wait(srv, [r1, r2])
        res1, res2 = srv.result(r1, config=False), srv.result(r2, config=False)
        assert res1["status"] == 0 and res2["status"] == 0
        assert res2["start_ms"] >= res1["finish_ms"] - 1.0
        assert (res1["energy"], res1["step"], res1["sweep"], res1["slot"]) == _alone_best(g1, b1, 2048, 4, 1)
        assert (res2["energy"], res2["step"], res2["sweep"], res2["slot"]) == _alone_best(g2, b2, 8192, 2, 2)
        assert srv.release(r1) and srv.release(r2)
        with pytest.raises(B.PaError):
            srv.poll(r1)                                      # forgotten


def test_stalled_request_times_out_and_others_complete():
    require_gpu()
    reqs = [(wl.gnm(1000, 6000, seed=31), wl.linear_betas(0.1, 2.5, 40), 512, 2, 1),
            (wl.torus(30, seed=32), wl.linear_betas(0.1, 3.0, 400), 1024, 2, 2),
            (wl.gnp(400, 0.05, seed=33), wl.linear_betas(0.2, 2.0, 30), 256, 3, 3)]
    with B.Server(4 << 30, n_streams=4, steps_per_tick=2) as srv:
        ids = []
        for i, (g, betas, R, S, seed) in enumerate(reqs):
            rid = srv.submit(g, betas, R, S, seed, timeout_ms=1500.0 if i == 1 else 0.0)
            if i == 1:
                srv.hold(rid)   # its host-side job stalls from the start
            ids.append(rid)
        assert _wait(srv, ids)
        assert srv.poll(ids[1]) == B.PA_ETIMEOUT
        with pytest.raises(B.PaError) as e:
            srv.result(ids[1], config=False)
        assert e.value.code == B.PA_ETIMEOUT
        for i in (0, 2):
            g, betas, R, S, seed = reqs[i]
            r = srv.result(ids[i], config=False)
            assert r["status"] == 0
            assert (r["energy"], r["step"], r["sweep"], r["slot"]) == _alone_best(g, betas, R, S, seed)
        st = srv.stats()
        assert st["completed"] == 3 and st["running"] == 0 and st["bytes_in_use"] == 0
