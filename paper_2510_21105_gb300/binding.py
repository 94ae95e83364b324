"""Thin ctypes binding of libpa.so (include/pa.h): argument marshalling only.

Every step of the annealing runs in the library's CUDA kernels; this module
converts NumPy arrays to pointers, checks return codes and raises
``PaError``. There is no CPU fallback: if ``libpa.so`` has not been built the
first call raises. PyTorch is used only to hand the library a stream and,
optionally, its caching allocator for device memory.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpa.so")
_lib = None
_lock = threading.Lock()

PA_OK, PA_EINVAL, PA_ENOMEM, PA_ECUDA, PA_ETIMEOUT, PA_EBUSY, PA_ESTATE = 0, -1, -2, -3, -4, -5, -6
PA_VARIANT_I8, PA_VARIANT_MSC, PA_VARIANT_AUTO, PA_VARIANT_MSC_PAIR = 0, 1, 2, 3


class PaError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code}){': ' + detail if detail else ''}")


class pa_anneal_opts(C.Structure):
    _fields_ = [("variant", C.c_int32), ("field_bits", C.c_int32), ("nlm_period", C.c_int32),
                ("adaptive", C.c_int32), ("rho", C.c_double), ("adapt_J", C.c_int32),
                ("adapt_dbeta_max", C.c_double), ("beta_max", C.c_double),
                ("replicas_per_cta", C.c_int32), ("threads_per_cta", C.c_int32),
                ("stream", C.c_void_p), ("record_counts", C.c_int32), ("time_kernels", C.c_int32),
                ("nlm_kind", C.c_int32), ("nlm_block", C.c_int32), ("acc_lo", C.c_double),
                ("acc_hi", C.c_double), ("reheat_after", C.c_int32), ("reheat_back", C.c_int32),
                ("msc_no_split", C.c_int32)]


class pa_stats_t(C.Structure):
    _fields_ = [("attempts", C.c_int64), ("accepts", C.c_int64), ("steps_run", C.c_int32),
                ("n_colours", C.c_int32), ("max_degree", C.c_int32), ("kernel_launches", C.c_int32),
                ("sweep_launches", C.c_int32), ("variant", C.c_int32), ("anneal_ms", C.c_double),
                ("sweep_ms", C.c_double), ("t_best_ms", C.c_double), ("total_weight", C.c_int64),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64)]


class pa_step_arrays(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in
                ("beta", "emin", "A", "T", "o", "accepts", "lnZ", "sweep_emin", "nlm_pairs",
                 "nlm_flips", "jsel", "counts", "t_ms")]


class pa_peaks(C.Structure):
    _fields_ = [("int_ops_per_s", C.c_double), ("philox_words_per_s", C.c_double),
                ("smem_bytes_per_s", C.c_double), ("sms", C.c_int32)]


class pa_shard_step(C.Structure):
    _fields_ = [("A", C.c_double), ("T", C.c_uint64), ("P_base", C.c_uint64), ("new_lo", C.c_int32),
                ("new_hi", C.c_int32), ("send", C.c_int32 * 64), ("recv", C.c_int32 * 64)]


class pa_job(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("betas", C.c_void_p), ("K", C.c_int32), ("R", C.c_int32),
                ("sweeps", C.c_int32), ("seed", C.c_uint64), ("opts", pa_anneal_opts)]


class pa_batch_opts(C.Structure):
    _fields_ = [("n_streams", C.c_int32), ("use_graph", C.c_int32), ("stream", C.c_void_p)]


class pa_request(C.Structure):
    _fields_ = [("n", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("w", C.c_void_p),
                ("betas", C.c_void_p), ("K", C.c_int32), ("R", C.c_int32), ("sweeps", C.c_int32),
                ("seed", C.c_uint64), ("opts", pa_anneal_opts), ("timeout_ms", C.c_double)]


class pa_response(C.Structure):
    _fields_ = [("cut", C.c_int64), ("energy", C.c_int32), ("step", C.c_int32), ("sweep", C.c_int32),
                ("slot", C.c_int32), ("status", C.c_int32), ("attempts", C.c_int64),
                ("submit_ms", C.c_double), ("start_ms", C.c_double), ("finish_ms", C.c_double)]


class pa_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("queued", C.c_int64), ("running", C.c_int64), ("bytes_in_use", C.c_int64),
                ("attempts", C.c_int64), ("elapsed_ms", C.c_double)]


class pa_resample_result(C.Structure):
    _fields_ = [("A", C.c_double), ("T", C.c_uint64), ("emin", C.c_int32), ("o", C.c_uint32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def lib():
    """Load libpa.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2510_21105_gb300.build` (CUDA is required; "
                                   "there is no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            sig = {
                "pa_version": ([], i32),
                "pa_strerror": ([C.c_int], C.c_char_p),
                "pa_last_error": ([vp], C.c_char_p),
                "pa_default_opts": ([C.POINTER(pa_anneal_opts)], None),
                "pa_create": ([C.POINTER(vp), i32, vp, vp, vp], C.c_int),
                "pa_destroy": ([vp], None),
                "pa_anneal": ([vp, vp, i32, i32, i32, u64, C.POINTER(pa_anneal_opts)], C.c_int),
                "pa_anneal_begin": ([vp, vp, i32, i32, i32, u64, C.POINTER(pa_anneal_opts)], C.c_int),
                "pa_anneal_run": ([vp, i32], C.c_int),
                "pa_sync": ([vp], C.c_int),
                "pa_best": ([vp, C.POINTER(i64), vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
                "pa_best_record": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)],
                                   C.c_int),
                "pa_get_state": ([vp, vp, vp], C.c_int),
                "pa_set_state": ([vp, vp, i32], C.c_int),
                "pa_energies": ([vp, vp, i32, vp, vp], C.c_int),
                "pa_save": ([vp, C.c_char_p], C.c_int),
                "pa_load": ([vp, C.c_char_p], C.c_int),
                "pa_stats": ([vp, C.POINTER(pa_stats_t)], C.c_int),
                "pa_run_info": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)],
                                C.c_int),
                "pa_step_stats": ([vp, C.POINTER(pa_step_arrays)], C.c_int),
                "pa_tables": ([vp, i32, vp, vp], C.c_int),
                "pa_colouring": ([vp, vp, vp], C.c_int),
                "pa_set_allocator": ([ALLOC_FN, FREE_FN, vp], None),
                "pa_resample_noalloc": ([vp, i32, dbl, dbl, u64, i32, vp, vp, C.POINTER(pa_resample_result),
                                         vp], C.c_int),
                "pa_batch_anneal": ([C.POINTER(pa_job), i32, C.POINTER(pa_batch_opts), C.POINTER(dbl)], C.c_int),
                "pa_server_start": ([C.POINTER(vp), C.c_size_t, i32, i32], C.c_int),
                "pa_server_submit": ([vp, C.POINTER(pa_request), C.POINTER(u64)], C.c_int),
                "pa_server_poll": ([vp, u64, C.POINTER(i32)], C.c_int),
                "pa_server_result": ([vp, u64, C.POINTER(pa_response), vp], C.c_int),
                "pa_server_stats": ([vp, C.POINTER(pa_server_stats_t)], C.c_int),
                "pa_server_release": ([vp, u64], C.c_int),
                "pa_probe_peaks": ([C.POINTER(pa_peaks), vp], C.c_int),
                "pa_shard_scratch_bytes": ([i32], C.c_size_t),
                "pa_shard_min": ([vp, i32, vp, C.POINTER(i32), vp], C.c_int),
                "pa_shard_partials": ([vp, i32, i32, dbl, dbl, vp, C.POINTER(dbl), C.POINTER(u64), vp], C.c_int),
                "pa_shard_plan": ([i32, i32, i32, vp, vp, C.c_uint32, C.POINTER(pa_shard_step)], C.c_int),
                "pa_shard_parents": ([vp, i32, i32, C.c_uint32, C.POINTER(pa_shard_step), vp, vp, vp], C.c_int),
                "pa_shard_gather": ([vp, vp, i32, vp, i32, vp, vp, vp], C.c_int),
                "pa_resample_offset": ([u64, i32], C.c_uint32),
                "pa_server_hold": ([vp, u64, i32], C.c_int),
                "pa_server_stop": ([vp], C.c_int),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
        return _lib


def exported_symbols():
    """Names declared in include/pa.h that the loaded library must export."""
    return ["pa_version", "pa_strerror", "pa_last_error", "pa_default_opts", "pa_create",
            "pa_destroy", "pa_anneal", "pa_anneal_begin", "pa_anneal_run", "pa_sync", "pa_best",
            "pa_best_record", "pa_get_state", "pa_set_state", "pa_energies", "pa_save", "pa_load", "pa_stats",
            "pa_step_stats", "pa_tables", "pa_colouring", "pa_set_allocator", "pa_run_info",
            "pa_resample_noalloc", "pa_batch_anneal", "pa_server_start", "pa_server_submit",
            "pa_server_poll", "pa_server_result", "pa_server_stats", "pa_server_stop",
            "pa_server_release", "pa_server_hold", "pa_probe_peaks", "pa_shard_scratch_bytes", "pa_shard_min",
            "pa_shard_partials", "pa_shard_plan", "pa_shard_parents", "pa_shard_gather", "pa_resample_offset"]


def strerror(code: int) -> str:
    try:
        return lib().pa_strerror(code).decode()
    except RuntimeError:
        return str(code)


def _check(rc: int, where: str, ctx=None):
    if rc != PA_OK:
        detail = lib().pa_last_error(ctx).decode() if ctx else ""
        raise PaError(rc, where, detail)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def pa_default_opts(**kw) -> pa_anneal_opts:
    o = pa_anneal_opts()
    lib().pa_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def pa_create(n: int, row_ptr, col, w=None):
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    cl = np.ascontiguousarray(col, dtype=np.uint16)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.int8)
    if len(rp) != n + 1:
        raise ValueError("row_ptr must have n + 1 entries")
    out = C.c_void_p()
    _check(lib().pa_create(C.byref(out), int(n), _ptr(rp), _ptr(cl), _ptr(ww)), "pa_create")
    return out


def pa_destroy(ctx):
    lib().pa_destroy(ctx)


def _betas(betas):
    return None if betas is None else np.ascontiguousarray(betas, dtype=np.float64)


def pa_anneal(ctx, betas, K: int, R: int, sweeps: int, seed: int, opts: pa_anneal_opts | None = None):
    b = _betas(betas)
    _check(lib().pa_anneal(ctx, _ptr(b), int(K), int(R), int(sweeps), int(seed) & (2**64 - 1),
                           C.byref(opts) if opts is not None else None), "pa_anneal", ctx)


def pa_anneal_begin(ctx, betas, K: int, R: int, sweeps: int, seed: int, opts: pa_anneal_opts | None = None):
    b = _betas(betas)
    _check(lib().pa_anneal_begin(ctx, _ptr(b), int(K), int(R), int(sweeps), int(seed) & (2**64 - 1),
                                 C.byref(opts) if opts is not None else None), "pa_anneal_begin", ctx)


def pa_anneal_run(ctx, k_end: int):
    _check(lib().pa_anneal_run(ctx, int(k_end)), "pa_anneal_run", ctx)


def pa_sync(ctx):
    _check(lib().pa_sync(ctx), "pa_sync", ctx)


def pa_best(ctx, n: int):
    cut = C.c_int64()
    step = C.c_int32()
    sweep = C.c_int32()
    cfg = np.zeros(n, np.int8)
    _check(lib().pa_best(ctx, C.byref(cut), _ptr(cfg), C.byref(step), C.byref(sweep)), "pa_best", ctx)
    return cut.value, cfg, step.value, sweep.value


def pa_best_record(ctx):
    v = [C.c_int32() for _ in range(4)]
    _check(lib().pa_best_record(ctx, *[C.byref(x) for x in v]), "pa_best_record", ctx)
    return tuple(x.value for x in v)


def pa_get_state(ctx, R: int, n: int):
    spins = np.zeros((R, n), np.int8)
    E = np.zeros(R, np.int32)
    _check(lib().pa_get_state(ctx, _ptr(spins), _ptr(E)), "pa_get_state", ctx)
    return spins, E


def pa_set_state(ctx, spins, steps_done: int):
    s = np.ascontiguousarray(spins, dtype=np.int8)
    _check(lib().pa_set_state(ctx, _ptr(s), int(steps_done)), "pa_set_state", ctx)


def pa_energies(ctx, spins, n: int):
    """Energies and cuts of host configurations (one per row), on the device."""
    s = np.ascontiguousarray(spins, dtype=np.int8)
    if s.ndim == 1:
        s = s.reshape(1, -1)
    if s.shape[1] != n:
        raise ValueError(f"configurations must have {n} spins, got {s.shape[1]}")
    R = s.shape[0]
    E = np.zeros(R, np.int32)
    cuts = np.zeros(R, np.int64)
    _check(lib().pa_energies(ctx, _ptr(s), int(R), _ptr(E), _ptr(cuts)), "pa_energies", ctx)
    return E, cuts


def pa_save(ctx, path: str):
    _check(lib().pa_save(ctx, path.encode()), "pa_save", ctx)


def pa_load(ctx, path: str):
    _check(lib().pa_load(ctx, path.encode()), "pa_load", ctx)


def pa_run_info(ctx):
    v = [C.c_int32() for _ in range(4)]
    _check(lib().pa_run_info(ctx, *[C.byref(x) for x in v]), "pa_run_info", ctx)
    return dict(R=v[0].value, K=v[1].value, S=v[2].value, steps_done=v[3].value)


def pa_stats(ctx) -> dict:
    st = pa_stats_t()
    _check(lib().pa_stats(ctx, C.byref(st)), "pa_stats", ctx)
    return {name: getattr(st, name) for name, _ in pa_stats_t._fields_}


def pa_step_stats(ctx, steps: int, R: int, S: int, counts: bool = False) -> dict:
    arrs = dict(beta=np.zeros(steps), emin=np.zeros(steps, np.int32), A=np.zeros(steps),
                T=np.zeros(steps, np.uint64), o=np.zeros(steps, np.uint32),
                accepts=np.zeros(steps, np.int64), lnZ=np.zeros(steps),
                sweep_emin=np.zeros((steps, max(S, 1)), np.int32),
                nlm_pairs=np.zeros(steps, np.int32), nlm_flips=np.zeros(steps, np.int64),
                jsel=np.zeros(steps, np.int32), t_ms=np.zeros(steps))
    if counts:
        arrs["counts"] = np.zeros((steps, R), np.int32)
    sa = pa_step_arrays()
    for k, v in arrs.items():
        setattr(sa, k, v.ctypes.data)
    _check(lib().pa_step_stats(ctx, C.byref(sa)), "pa_step_stats", ctx)
    arrs["sweep_emin"] = arrs["sweep_emin"][:, :S]
    return arrs


def pa_tables(ctx, k: int, maxdeg: int):
    acc = np.zeros(maxdeg + 1, np.uint32)
    q = np.zeros(32, np.float64)
    _check(lib().pa_tables(ctx, int(k), _ptr(acc), _ptr(q)), "pa_tables", ctx)
    return acc, q


def pa_colouring(ctx, n: int):
    colour = np.zeros(n, np.int32)
    pos = np.zeros(n, np.int32)
    rc = lib().pa_colouring(ctx, _ptr(colour), _ptr(pos))
    if rc < 0:
        _check(rc, "pa_colouring", ctx)
    return rc, colour, pos


def pa_resample_noalloc(energies_ptr: int, R: int, beta_prev: float, beta_k: float, seed: int, k: int,
                        parent_ptr: int, counts_ptr: int | None = None, stream=None, want_result: bool = True):
    """Resampling step with caller-owned device buffers and no device allocation
    (see include/pa.h); pointers are raw device addresses. With
    want_result=False the host result is not requested (NULL is passed), so
    the call only enqueues its kernel and returns None."""
    res = pa_resample_result() if want_result else None
    _check(lib().pa_resample_noalloc(C.c_void_p(energies_ptr), int(R), float(beta_prev), float(beta_k),
                                     int(seed) & (2**64 - 1), int(k), C.c_void_p(parent_ptr),
                                     C.c_void_p(counts_ptr) if counts_ptr else None,
                                     C.byref(res) if want_result else None, stream), "pa_resample_noalloc")
    return dict(A=res.A, T=res.T, emin=res.emin, o=res.o) if want_result else None


def pa_batch_anneal(items, n_streams: int = 0, use_graph: bool = False, stream=None) -> float:
    """Run many anneals together (see include/pa.h). items: list of
    (Annealer, betas, R, S, seed, K, opts-dict). Returns the device time in ms."""
    arr = (pa_job * len(items))()
    keep = []
    for i, (ann, betas, R, S, seed, K, kw) in enumerate(items):
        b = _betas(betas)
        keep.append(b)
        K = len(b) if (K is None and b is not None) else K
        o = pa_default_opts(**(kw or {}))
        arr[i] = pa_job(ann.ctx, None if b is None else b.ctypes.data, int(K), int(R), int(S),
                        int(seed) & (2**64 - 1), o)
        ann.R, ann.S, ann.K = R, S, K
    bo = pa_batch_opts(int(n_streams), int(bool(use_graph)), stream)
    ms = C.c_double(0.0)
    rc = lib().pa_batch_anneal(arr, len(items), C.byref(bo), C.byref(ms))
    if rc != PA_OK:
        detail = ""
        for ann, *_ in items:
            d = lib().pa_last_error(ann.ctx).decode()
            if d:
                detail = d
                break
        raise PaError(rc, "pa_batch_anneal", detail)
    return ms.value


class Server:
    """Continuous-batching request loop (pa_server_*): submit anneal requests,
    poll, and read results; device memory is admitted against hbm_budget."""

    def __init__(self, hbm_budget: int, n_streams: int = 16, steps_per_tick: int = 8):
        self.h = C.c_void_p()
        _check(lib().pa_server_start(C.byref(self.h), int(hbm_budget), int(n_streams), int(steps_per_tick)),
               "pa_server_start")
        self.n = {}

    def submit(self, g, betas, R: int, S: int, seed: int, K: int | None = None, timeout_ms: float = 0.0,
               **opts) -> int:
        rp = g.rp_u32
        col = g.col_u16
        w = None if g.w is None else np.ascontiguousarray(g.w, np.int8)
        b = _betas(betas)
        if K is None:
            K = len(b) if b is not None else 0
        req = pa_request(int(g.n), rp.ctypes.data, col.ctypes.data if len(col) else None,
                         None if w is None else w.ctypes.data, None if b is None else b.ctypes.data,
                         int(K), int(R), int(S), int(seed) & (2**64 - 1), pa_default_opts(**opts),
                         float(timeout_ms))
        rid = C.c_uint64()
        _check(lib().pa_server_submit(self.h, C.byref(req), C.byref(rid)), "pa_server_submit")
        self.n[rid.value] = g.n
        return rid.value

    def poll(self, rid: int) -> int:
        st = C.c_int32()
        _check(lib().pa_server_poll(self.h, int(rid), C.byref(st)), "pa_server_poll")
        return st.value

    def result(self, rid: int, config: bool = True):
        r = pa_response()
        cfg = np.zeros(self.n[rid], np.int8) if config else None
        rc = lib().pa_server_result(self.h, int(rid), C.byref(r), _ptr(cfg))
        if rc == PA_EBUSY:
            return None
        _check(rc, "pa_server_result")
        out = {name: getattr(r, name) for name, _ in pa_response._fields_}
        out["config"] = cfg
        return out

    def release(self, rid: int) -> bool:
        """Forget a finished request; False if it has not finished yet."""
        rc = lib().pa_server_release(self.h, int(rid))
        if rc == PA_EBUSY:
            return False
        _check(rc, "pa_server_release")
        self.n.pop(rid, None)
        return True

    def hold(self, rid: int, hold: bool = True):
        """Testing hook: stop (or resume) enqueuing the request's steps."""
        _check(lib().pa_server_hold(self.h, int(rid), int(bool(hold))), "pa_server_hold")

    def stats(self) -> dict:
        st = pa_server_stats_t()
        _check(lib().pa_server_stats(self.h, C.byref(st)), "pa_server_stats")
        return {name: getattr(st, name) for name, _ in pa_server_stats_t._fields_}

    def stop(self):
        if self.h:
            _check(lib().pa_server_stop(self.h), "pa_server_stop")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()


_alloc_refs = None


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_refs
    if not enable:
        lib().pa_set_allocator(ALLOC_FN(0), FREE_FN(0), None)
        _alloc_refs = None
        return
    import torch

    def _alloc(nbytes, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:   # out of memory: the library reports PA_ENOMEM
            return None

    def _free(ptr, _user):
        torch.cuda.caching_allocator_delete(ptr)

    _alloc_refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    lib().pa_set_allocator(_alloc_refs[0], _alloc_refs[1], None)


def probe_peaks(stream=None) -> dict:
    """Integer, Philox and shared-memory throughput of the current device
    (pa_probe_peaks), the roofline denominators of the sweep."""
    p = pa_peaks()
    _check(lib().pa_probe_peaks(C.byref(p), stream), "pa_probe_peaks")
    return {name: getattr(p, name) for name, _ in pa_peaks._fields_}


def current_stream_handle():
    """cudaStream_t of torch's current stream (the library launches there)."""
    import torch

    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Annealer:
    """Owns one pa_ctx for a graph given as CSR arrays (see workloads.Graph)."""

    def __init__(self, n, rp, col, w=None):
        self.n = int(n)
        self.ctx = pa_create(self.n, rp, col, w)
        self.R = self.S = self.K = 0

    @classmethod
    def from_graph(cls, g):
        return cls(g.n, g.rp_u32, g.col_u16, g.w)

    def close(self):
        if self.ctx:
            pa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _opts(self, kw):
        stream = kw.pop("stream", None)
        o = pa_default_opts(**kw)
        if stream is not None:
            o.stream = stream
        return o

    def anneal(self, betas, R, S, seed, K=None, **kw):
        K = len(betas) if K is None else K
        self.R, self.S, self.K = R, S, K
        pa_anneal(self.ctx, betas, K, R, S, seed, self._opts(kw))

    def begin(self, betas, R, S, seed, K=None, **kw):
        K = len(betas) if K is None else K
        self.R, self.S, self.K = R, S, K
        pa_anneal_begin(self.ctx, betas, K, R, S, seed, self._opts(kw))

    def run(self, k_end):
        pa_anneal_run(self.ctx, k_end)

    def sync(self):
        pa_sync(self.ctx)

    def best(self):
        return pa_best(self.ctx, self.n)

    def best_record(self):
        return pa_best_record(self.ctx)

    def state(self):
        return pa_get_state(self.ctx, self.R, self.n)

    def set_state(self, spins, steps_done):
        pa_set_state(self.ctx, spins, steps_done)

    def energies(self, spins):
        return pa_energies(self.ctx, spins, self.n)

    def stats(self):
        return pa_stats(self.ctx)

    def step_stats(self, counts=False):
        st = self.stats()
        return pa_step_stats(self.ctx, st["steps_run"], self.R, self.S, counts)

    def tables(self, k, maxdeg):
        return pa_tables(self.ctx, k, maxdeg)

    def colouring(self):
        return pa_colouring(self.ctx, self.n)

    def save(self, path):
        pa_save(self.ctx, path)

    def load(self, path):
        pa_load(self.ctx, path)
        info = pa_run_info(self.ctx)
        self.R, self.K, self.S = info["R"], info["K"], info["S"]
