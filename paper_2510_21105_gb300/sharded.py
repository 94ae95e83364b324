"""Resampling of one population split over the ranks of a torch.distributed
group (replica sharding across GPUs): the driver of the pa_shard_* entry
points of include/pa.h.

Rank g of G holds the slots [g R/G, (g+1) R/G) of a population of R = 2^a
replicas (spins int8 [R/G][ncols], energies int32 [R/G], device tensors). One
temperature step's resampling, with the same arithmetic as the resampling
inside pa_anneal (Sec. 3: population annealing; weights, pairwise weight sum A,
integer weights and systematic copies as the library defines them):

  1. E_min,g on the device, all-reduce min;
  2. weights, the rank's subtree sum A_g and integer total T_g on the device;
     all-gather of (A_g, T_g);
  3. pa_shard_plan on the host: A (bitwise the single-population sum: the rank
     subtrees are combined in the tree's own order), T, the contiguous new
     slots this rank's parents fill and the rows exchanged with every rank;
  4. parents of those slots and the rows gathered in new-slot order on the
     device; one all-to-all moves them to their owners.

Every output (copy counts, parents, A, T, the new population) equals the
single-population resampling bit for bit. The local arithmetic is pluggable:
``LibraryShard`` runs it in the library's CUDA kernels; a test may supply
another implementation with the same methods to exercise the exchange on CPU
ranks. There are no other data-path collectives: sweeps and best tracking act
on each rank's replicas alone (all randomness is keyed by the global slot).
"""
from __future__ import annotations

import ctypes as C
import struct

from . import binding as B


def shard_range(R: int, G: int, g: int):
    """Slots [lo, hi) of rank g (R and G powers of two, G <= R)."""
    if R < 1 or G < 1 or R & (R - 1) or G & (G - 1) or G > R or not 0 <= g < G:
        raise ValueError(f"sharding needs R and G powers of two with G <= R (R={R}, G={G}, g={g})")
    w = R // G
    return g * w, (g + 1) * w


def plan(G: int, g: int, R: int, A_all, T_all, o: int) -> dict:
    """Host plan of the step (pa_shard_plan): A, T, the new slots this rank's
    parents fill, and per-rank send / receive row counts."""
    A = (C.c_double * G)(*[float(a) for a in A_all])
    T = (C.c_uint64 * G)(*[int(t) for t in T_all])
    st = B.pa_shard_step()
    B._check(B.lib().pa_shard_plan(int(G), int(g), int(R), C.cast(A, C.c_void_p), C.cast(T, C.c_void_p),
                                   int(o) & 0xFFFFFFFF, C.byref(st)), "pa_shard_plan")
    return dict(A=st.A, T=st.T, P_base=st.P_base, new_lo=st.new_lo, new_hi=st.new_hi,
                send=list(st.send[:G]), recv=list(st.recv[:G]))


def resample_offset(seed: int, k: int) -> int:
    """Offset word o of step k (word 0 of Philox(0, 0, k, tag 1))."""
    return int(B.lib().pa_resample_offset(int(seed) & (2**64 - 1), int(k)))


class LibraryShard:
    """Local arithmetic of a rank in the library's CUDA kernels (device tensors)."""

    def __init__(self, n_local: int, device, stream=None):
        import torch

        self.torch = torch
        self.n = int(n_local)
        self.device = device
        self.stream = stream
        self.scratch = torch.empty(int(B.lib().pa_shard_scratch_bytes(self.n)), dtype=torch.uint8, device=device)
        self.iscratch = torch.empty(4, dtype=torch.int32, device=device)

    def emin(self, E) -> int:
        out = C.c_int32()
        B._check(B.lib().pa_shard_min(E.data_ptr(), self.n, self.iscratch.data_ptr(), C.byref(out), self.stream),
                 "pa_shard_min")
        return out.value

    def partials(self, E, emin: int, beta_prev: float, beta_k: float):
        A, T = C.c_double(), C.c_uint64()
        B._check(B.lib().pa_shard_partials(E.data_ptr(), self.n, int(emin), float(beta_prev), float(beta_k),
                                           self.scratch.data_ptr(), C.byref(A), C.byref(T), self.stream),
                 "pa_shard_partials")
        return A.value, T.value

    def parents(self, R: int, o: int, step: dict):
        torch = self.torch
        st = B.pa_shard_step()
        st.A, st.T, st.P_base, st.new_lo, st.new_hi = step["A"], step["T"], step["P_base"], step["new_lo"], step["new_hi"]
        src = torch.empty(max(step["new_hi"] - step["new_lo"], 1), dtype=torch.int32, device=self.device)
        counts = torch.empty(self.n, dtype=torch.int32, device=self.device)
        B._check(B.lib().pa_shard_parents(self.scratch.data_ptr(), self.n, int(R), int(o) & 0xFFFFFFFF,
                                          C.byref(st), src.data_ptr(), counts.data_ptr(), self.stream),
                 "pa_shard_parents")
        return src[: step["new_hi"] - step["new_lo"]], counts

    def gather(self, spins, E, src):
        torch = self.torch
        nout = int(src.numel())
        out = torch.empty((nout, spins.shape[1]), dtype=torch.int8, device=self.device)
        eout = torch.empty(nout, dtype=torch.int32, device=self.device)
        B._check(B.lib().pa_shard_gather(spins.data_ptr(), E.data_ptr(), int(spins.shape[1]), src.data_ptr(), nout,
                                         out.data_ptr(), eout.data_ptr(), self.stream), "pa_shard_gather")
        return out, eout


def _f64_bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", float(x)))[0]


def _bits_f64(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", int(b)))[0]


class ShardedResampler:
    """The resampling step of one population spread over a process group.

    local: the rank's arithmetic (LibraryShard, or a test stand-in with the
    same methods); dist: torch.distributed (initialised); device: where the
    collectives' tensors live (cuda for NCCL, cpu for gloo)."""

    def __init__(self, R: int, local, dist, group=None, device="cpu"):
        self.R = int(R)
        self.dist = dist
        self.group = group
        self.G = dist.get_world_size(group)
        self.g = dist.get_rank(group)
        self.lo, self.hi = shard_range(self.R, self.G, self.g)
        self.local = local
        self.device = device

    def step(self, spins, E, beta_prev: float, beta_k: float, seed: int, k: int):
        """Resample from beta_prev to beta_k. spins [R/G][ncols] int8 and E
        [R/G] int32 are the rank's slots; returns the rank's new slots and a
        record (emin, A, T, o, the rank's copy counts)."""
        import torch

        dist = self.dist
        emin = torch.tensor([self.local.emin(E)], dtype=torch.int64, device=self.device)
        dist.all_reduce(emin, op=dist.ReduceOp.MIN, group=self.group)
        emin = int(emin.item())
        A_g, T_g = self.local.partials(E, emin, beta_prev, beta_k)
        mine = torch.tensor([_f64_bits(A_g), int(T_g)], dtype=torch.int64, device=self.device)
        every = [torch.zeros(2, dtype=torch.int64, device=self.device) for _ in range(self.G)]
        dist.all_gather(every, mine, group=self.group)
        A_all = [_bits_f64(int(t[0].item())) for t in every]
        T_all = [int(t[1].item()) for t in every]
        o = resample_offset(seed, k)
        p = plan(self.G, self.g, self.R, A_all, T_all, o)
        src, counts = self.local.parents(self.R, o, p)
        rows, erows = self.local.gather(spins, E, src)
        n_local = self.hi - self.lo
        new_spins = torch.empty((n_local, spins.shape[1]), dtype=torch.int8, device=rows.device)
        new_E = torch.empty(n_local, dtype=torch.int32, device=rows.device)
        if self.G == 1:
            new_spins.copy_(rows)
            new_E.copy_(erows)
        else:
            dist.all_to_all_single(new_spins, rows, p["recv"], p["send"], group=self.group)
            dist.all_to_all_single(new_E, erows, p["recv"], p["send"], group=self.group)
        rec = dict(emin=emin, A=p["A"], T=p["T"], o=o, counts=counts, new_lo=p["new_lo"], new_hi=p["new_hi"])
        return new_spins, new_E, rec


__all__ = ["ShardedResampler", "LibraryShard", "plan", "shard_range", "resample_offset"]
