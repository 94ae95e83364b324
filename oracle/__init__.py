"""CPU oracle for Population Annealing Monte Carlo on Max-Cut (ctypes wrapper).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(``paper_2510_21105_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``pamc_oracle.c`` (plain single-threaded C, built with
``-O2 -ffp-contract=off``); this module only builds it with gcc and marshals
NumPy arrays. Paper references: Eq. 1 (Max-Cut objective), Sec. 2 (Ising
mapping), Sec. 3 (PAMC with adaptive stochasticity and non-local moves).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pamc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpamc_oracle.so")
_lock = threading.Lock()
_lib = None


_LIB_OMP = os.path.join(_HERE, "_build", "libpamc_oracle_omp.so")
_lib_omp = None


def _compile(out: str, extra, force: bool) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (single-threaded, no FMA contraction)."""
    return _compile(_LIB, [], force)


def build_parallel(force: bool = False) -> str:
    """The same source built with OpenMP: replicas swept on several threads
    between resamplings. For timing only; results equal the checking build."""
    return _compile(_LIB_OMP, ["-fopenmp"], force)


class OrcOpts(C.Structure):
    _fields_ = [("nlm_period", C.c_int32), ("adaptive", C.c_int32), ("rho", C.c_double),
                ("adapt_J", C.c_int32), ("adapt_dbeta_max", C.c_double), ("beta_max", C.c_double),
                ("nlm_kind", C.c_int32), ("nlm_block", C.c_int32), ("acc_lo", C.c_double),
                ("acc_hi", C.c_double), ("reheat_after", C.c_int32), ("reheat_back", C.c_int32)]


class OrcOut(C.Structure):
    _fields_ = [("spins", C.c_void_p), ("E", C.c_void_p), ("step_beta", C.c_void_p),
                ("step_emin", C.c_void_p), ("step_A", C.c_void_p), ("step_T", C.c_void_p),
                ("step_o", C.c_void_p), ("step_accepts", C.c_void_p), ("step_lnZ", C.c_void_p),
                ("step_counts", C.c_void_p), ("step_sweep_emin", C.c_void_p),
                ("step_nlm_pairs", C.c_void_p), ("step_nlm_flips", C.c_void_p),
                ("step_jsel", C.c_void_p), ("best_config", C.c_void_p),
                ("best", C.c_int32 * 4), ("steps_run", C.c_int32)]


def _declare(L):
    """Argument and result types of the oracle's C functions."""
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    L.orc_philox4x32_10.argtypes = [vp, vp, vp]
    L.orc_energy.argtypes = [i32, vp, vp, vp, vp]
    L.orc_energy.restype = i64
    L.orc_total_weight.argtypes = [i32, vp, vp, vp]
    L.orc_total_weight.restype = i64
    L.orc_greedy_colour.argtypes = [i32, vp, vp, vp]
    L.orc_greedy_colour.restype = i32
    L.orc_accept_table.argtypes = [dbl, i32, vp]
    L.orc_resample.argtypes = [i32, vp, dbl, C.c_uint32, vp, vp, vp, vp, vp]
    L.orc_resample.restype = C.c_int
    L.orc_houdayer_pair.argtypes = [i32, vp, vp, vp, vp, C.c_uint32, vp]
    L.orc_houdayer_pair.restype = i32
    L.orc_nlm_order.argtypes = [i32, u64, i32, vp]
    L.orc_anneal.argtypes = [i32, vp, vp, vp, vp, i32, i32, i32, u64, C.POINTER(OrcOpts),
                             C.POINTER(OrcOut)]
    L.orc_anneal.restype = C.c_int
    L.orc_step.argtypes = [i32, vp, vp, vp, i32, i32, u64, i32, dbl, dbl, i32, i32, vp, i32,
                           vp, vp, vp, vp, vp]
    L.orc_block_move.argtypes = [i32, vp, vp, vp, vp, vp, i32, dbl, i32, C.c_uint32, vp]
    L.orc_block_move.restype = i32
    L.orc_step.restype = C.c_int
    L.orc_sweep_uniforms.argtypes = [u64, i32, vp, vp, i32, i32, vp]
    L.orc_shard_partials.argtypes = [i32, vp, i32, dbl, C.POINTER(dbl), C.POINTER(u64), vp]
    L.orc_systematic_count.argtypes = [u64, i32, u64, C.c_uint32]
    L.orc_systematic_count.restype = i64
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
        return _lib


def lib_parallel(threads: int = 0):
    """The OpenMP timing build (threads > 0 sets its thread count)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            _lib_omp = _declare(C.CDLL(build_parallel()))
            _lib_omp.orc_threads.argtypes = [C.c_int32]
            _lib_omp.orc_threads.restype = C.c_int
    if threads:
        _lib_omp.orc_threads(int(threads))
    return _lib_omp


def parallel_threads() -> int:
    return int(lib_parallel().orc_threads(0))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _graph_arrays(rp, col, w):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.int8)
    return rp, col, w


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def sweep_uniforms(seed: int, vertices, slots, k: int, s: int):
    """The 32-bit uniforms of Metropolis attempts (vertex, replica) at step k,
    sweep s (``orc_sweep_uniforms``)."""
    i = np.ascontiguousarray(vertices, dtype=np.int32)
    r = np.ascontiguousarray(slots, dtype=np.int32)
    u = np.zeros(len(i), np.uint32)
    lib().orc_sweep_uniforms(int(seed), len(i), _p(i), _p(r), int(k), int(s), _p(u))
    return u


def energy(rp, col, w, x) -> int:
    rp, col, w = _graph_arrays(rp, col, w)
    x = np.ascontiguousarray(x, dtype=np.int8)
    return int(lib().orc_energy(len(rp) - 1, _p(rp), _p(col), _p(w), _p(x)))


def total_weight(rp, col, w) -> int:
    rp, col, w = _graph_arrays(rp, col, w)
    return int(lib().orc_total_weight(len(rp) - 1, _p(rp), _p(col), _p(w)))


def greedy_colour(rp, col):
    rp, col, _ = _graph_arrays(rp, col, None)
    n = len(rp) - 1
    colour = np.zeros(max(n, 1), np.int32)
    ncol = lib().orc_greedy_colour(n, _p(rp), _p(col), _p(colour))
    return int(ncol), colour[:n]


def accept_table(beta: float, mmax: int):
    T = np.zeros(mmax + 1, np.uint32)
    lib().orc_accept_table(float(beta), int(mmax), _p(T))
    return T


def resample(E, q: float, o: int):
    E = np.ascontiguousarray(E, dtype=np.int32)
    R = len(E)
    counts = np.zeros(R, np.int32)
    parent = np.zeros(R, np.int32)
    emin = C.c_int32()
    A = C.c_double()
    T = C.c_uint64()
    rc = lib().orc_resample(R, _p(E), float(q), int(o), _p(counts), _p(parent), C.byref(emin),
                            C.byref(A), C.byref(T))
    if rc != 0:
        raise ValueError(f"orc_resample failed: {rc}")
    return dict(counts=counts, parent=parent, emin=emin.value, A=A.value, T=T.value)


def shard_partials(E, emin: int, q: float):
    """Weights of one shard with the population's E_min given: (A, T, t)
    (``orc_shard_partials``)."""
    E = np.ascontiguousarray(E, dtype=np.int32)
    t = np.zeros(len(E), np.uint64)
    A, T = C.c_double(), C.c_uint64()
    lib().orc_shard_partials(len(E), _p(E), int(emin), float(q), C.byref(A), C.byref(T), _p(t))
    return A.value, T.value, t


def systematic_count(P: int, R: int, T: int, o: int) -> int:
    """F(P) of systematic resampling (``orc_systematic_count``)."""
    return int(lib().orc_systematic_count(int(P), int(R), int(T), int(o)))


def houdayer_pair(rp, col, xa, xb, u: int):
    rp, col, _ = _graph_arrays(rp, col, None)
    xa = np.array(xa, dtype=np.int8)
    xb = np.array(xb, dtype=np.int8)
    n = len(rp) - 1
    cl = np.zeros(n, np.uint8)
    size = lib().orc_houdayer_pair(n, _p(rp), _p(col), _p(xa), _p(xb), int(u), _p(cl))
    return int(size), xa, xb, cl.astype(bool)


def block_move(rp, col, w, x, E: int, b: int, q: float, seed_vertex: int, u: int):
    """One block move on a copy of x (``orc_block_move``): returns (size
    flipped or 0, new spins, new energy, block mask)."""
    rp, col, w = _graph_arrays(rp, col, w)
    x = np.array(x, dtype=np.int8)
    n = len(rp) - 1
    e = C.c_int32(int(E))
    mask = np.zeros(n, np.uint8)
    size = lib().orc_block_move(n, _p(rp), _p(col), _p(w), _p(x), C.byref(e), int(b), float(q),
                                int(seed_vertex), int(u), _p(mask))
    return int(size), x, int(e.value), mask.astype(bool)


def nlm_order(R: int, seed: int, k: int):
    order = np.zeros(R, np.int32)
    lib().orc_nlm_order(int(R), int(seed), int(k), _p(order))
    return order


@dataclass
class AnnealResult:
    spins: np.ndarray
    E: np.ndarray
    step_beta: np.ndarray
    step_emin: np.ndarray
    step_A: np.ndarray
    step_T: np.ndarray
    step_o: np.ndarray
    step_accepts: np.ndarray
    step_lnZ: np.ndarray
    step_sweep_emin: np.ndarray
    step_nlm_pairs: np.ndarray
    step_nlm_flips: np.ndarray
    step_jsel: np.ndarray
    best_config: np.ndarray
    best_E: int
    best_step: int
    best_sweep: int
    best_slot: int
    steps_run: int
    step_counts: np.ndarray | None = field(default=None)


def anneal(rp, col, w, betas, R: int, S: int, seed: int, *, K: int | None = None,
           nlm_period: int = 0, adaptive: int = 0, rho: float = 0.5, adapt_J: int = 8,
           adapt_dbeta_max: float = 0.05, beta_max: float = 0.0, record_counts: bool = False,
           nlm_kind: int = 0, nlm_block: int = 1, acc_lo: float = 0.0, acc_hi: float = 1.0,
           reheat_after: int = 0, reheat_back: int = 0, parallel: bool = False):
    """Run the oracle PAMC (see ``orc_anneal`` in pamc_oracle.c). parallel:
    the OpenMP timing build (same results)."""
    rp, col, w = _graph_arrays(rp, col, w)
    n = len(rp) - 1
    if adaptive:
        if K is None:
            raise ValueError("adaptive mode needs K (maximum number of steps)")
        b = None
    else:
        b = np.ascontiguousarray(betas, dtype=np.float64)
        K = len(b) if K is None else K
    opts = OrcOpts(int(nlm_period), int(adaptive), float(rho), int(adapt_J),
                   float(adapt_dbeta_max), float(beta_max), int(nlm_kind), int(nlm_block), float(acc_lo),
                   float(acc_hi), int(reheat_after), int(reheat_back))
    arr = dict(
        spins=np.zeros((R, n), np.int8), E=np.zeros(R, np.int32), step_beta=np.zeros(K),
        step_emin=np.zeros(K, np.int32), step_A=np.zeros(K), step_T=np.zeros(K, np.uint64),
        step_o=np.zeros(K, np.uint32), step_accepts=np.zeros(K, np.int64), step_lnZ=np.zeros(K),
        step_sweep_emin=np.zeros((K, max(S, 1)), np.int32), step_nlm_pairs=np.zeros(K, np.int32),
        step_nlm_flips=np.zeros(K, np.int64), step_jsel=np.full(K, -1, np.int32),
        best_config=np.zeros(n, np.int8))
    counts = np.zeros((K, R), np.int32) if record_counts else None
    out = OrcOut()
    for name, a in arr.items():
        setattr(out, name, a.ctypes.data)
    out.step_counts = counts.ctypes.data if counts is not None else None
    L = lib_parallel() if parallel else lib()
    rc = L.orc_anneal(n, _p(rp), _p(col), _p(w), _p(b), int(K), int(R), int(S), int(seed),
                          C.byref(opts), C.byref(out))
    if rc != 0:
        raise ValueError(f"orc_anneal rejected its arguments (rc={rc})")
    ks = out.steps_run
    res = AnnealResult(
        spins=arr["spins"], E=arr["E"], step_beta=arr["step_beta"][:ks],
        step_emin=arr["step_emin"][:ks], step_A=arr["step_A"][:ks], step_T=arr["step_T"][:ks],
        step_o=arr["step_o"][:ks], step_accepts=arr["step_accepts"][:ks],
        step_lnZ=arr["step_lnZ"][:ks], step_sweep_emin=arr["step_sweep_emin"][:ks, :S],
        step_nlm_pairs=arr["step_nlm_pairs"][:ks], step_nlm_flips=arr["step_nlm_flips"][:ks],
        step_jsel=arr["step_jsel"][:ks], best_config=arr["best_config"], best_E=out.best[0],
        best_step=out.best[1], best_sweep=out.best[2], best_slot=out.best[3], steps_run=ks,
        step_counts=None if counts is None else counts[:ks])
    return res


def step_replay(rp, col, w, spins_in, S: int, seed: int, k: int, beta_prev: float, beta_k: float,
                subset, nlm_now: bool = False, want_counts: bool = True, nlm_block: int = 0):
    """Replay temperature step k for the listed new slots (``orc_step``)."""
    rp, col, w = _graph_arrays(rp, col, w)
    spins_in = np.ascontiguousarray(spins_in, dtype=np.int8)
    R, n = spins_in.shape
    sub = np.ascontiguousarray(subset, dtype=np.int32)
    out = np.zeros((len(sub), n), np.int8)
    E = np.zeros(len(sub), np.int32)
    counts = np.zeros(R, np.int32) if want_counts else None
    acc = C.c_int64()
    rc = lib().orc_step(n, _p(rp), _p(col), _p(w), R, int(S), int(seed), int(k), float(beta_prev),
                        float(beta_k), int(bool(nlm_now)), int(nlm_block), _p(spins_in), len(sub),
                        _p(sub), _p(out),
                        _p(E), _p(counts), C.byref(acc))
    if rc != 0:
        raise ValueError(f"orc_step failed (rc={rc})")
    return dict(spins=out, E=E, counts=counts, accepts=acc.value)
