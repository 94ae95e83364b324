"""Seeded synthetic Max-Cut instances and annealing schedules.

This module holds input generation only: no energy, no random numbers of the
annealing method, no acceptance rule. It serves both the CUDA path and the
CPU oracle (which never share anything else), so every graph a test or the
benchmark uses comes from here.

The G-set instances the paper evaluates (Sec. 1: 800 to 20,000 nodes,
random / toroidal / planar topologies, unsigned or signed unit weights; G63:
N = 7000, M = 41,459, unweighted) are not available, so seeded stand-ins of
the same shapes are generated with NumPy's PCG64:

* ``gnp(n, p)``: every pair i < j joined independently with probability p.
* ``gnm(n, m)``: m distinct pairs drawn uniformly without replacement
  (G63-shaped at n = 7000, m = 41459).
* ``torus(L)``: L x L periodic grid, edges right and down, weights +-1 drawn
  equiprobably (G-set toroidal instances are signed).
* ``delaunay(n)``: Delaunay triangulation of n uniform points in the unit
  square (planar-like, unit weights).

Graphs are returned in CSR form with every undirected edge stored in both
rows and each row sorted by neighbour index.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    n: int
    rp: np.ndarray          # int64 [n+1] row pointers
    col: np.ndarray         # int32 [2M] neighbour indices
    w: np.ndarray | None    # int8 [2M] edge weights (+-1) or None (all +1)
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.rp[-1]) // 2

    @property
    def maxdeg(self) -> int:
        return int(np.diff(self.rp).max()) if self.n else 0

    @property
    def rp_u32(self) -> np.ndarray:
        return np.ascontiguousarray(self.rp, dtype=np.uint32)

    @property
    def col_u16(self) -> np.ndarray:
        if self.n > 65536:
            raise ValueError("uint16 column indices need n <= 65536")
        return np.ascontiguousarray(self.col, dtype=np.uint16)

    def edges(self):
        """Undirected edge list (i < j) with weights."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rp))
        keep = self.col > rows
        w = np.ones(int(keep.sum()), np.int8) if self.w is None else self.w[keep]
        return rows[keep], self.col[keep].astype(np.int64), w


def from_edges(n: int, i, j, w=None, name: str = "") -> Graph:
    """CSR from an undirected edge list (no self loops, no duplicates)."""
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    if np.any(i == j):
        raise ValueError("self loop")
    src = np.concatenate([i, j])
    dst = np.concatenate([j, i])
    ww = None if w is None else np.concatenate([np.asarray(w, np.int8)] * 2)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    if ww is not None:
        ww = ww[order]
    if len(src) > 1 and np.any((src[1:] == src[:-1]) & (dst[1:] == dst[:-1])):
        raise ValueError("duplicate edge")
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    return Graph(n=n, rp=rp, col=dst.astype(np.int32), w=ww, name=name)


def gnp(n: int, p: float, seed: int = 0) -> Graph:
    """Erdos-Renyi G(n, p): pair (i, j), i < j, in row-major order is joined
    iff its uniform draw is below p."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(len(iu)) < p
    return from_edges(n, iu[keep], ju[keep], name=f"gnp{n}_p{p}_s{seed}")


def gnm(n: int, m: int, seed: int = 0) -> Graph:
    """m distinct unordered pairs drawn uniformly without replacement
    (pairs drawn in batches; self loops and repeats rejected in draw order)."""
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")
    rng = np.random.Generator(np.random.PCG64(seed))
    seen: set = set()
    ei, ej = [], []
    while len(ei) < m:
        a = rng.integers(0, n, size=2 * (m - len(ei)) + 16)
        b = rng.integers(0, n, size=len(a))
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            key = (x, y) if x < y else (y, x)
            if key in seen:
                continue
            seen.add(key)
            ei.append(key[0])
            ej.append(key[1])
            if len(ei) == m:
                break
    return from_edges(n, ei, ej, name=f"gnm{n}_m{m}_s{seed}")


def gnp_sparse(n: int, p: float, seed: int = 0) -> Graph:
    """G(n, p) for large n: the edge count is drawn Binomial(n(n-1)/2, p),
    then that many distinct pairs uniformly (equal in law to G(n, p))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = int(rng.binomial(n * (n - 1) // 2, p))
    g = gnm(n, m, seed=int(rng.integers(0, 2**63 - 1)))
    g.name = f"gnp{n}_p{p:.6f}_s{seed}"
    return g


def torus(L: int, seed: int = 0, signed: bool = True) -> Graph:
    """L x L periodic grid in row-major order; vertex (r, c) joins (r, c+1)
    and (r+1, c) modulo L. Signed weights are +-1 with equal probability,
    drawn in that edge order."""
    if L < 3:
        raise ValueError("torus needs L >= 3 (no multi-edges)")
    r, c = np.divmod(np.arange(L * L), L)
    right = r * L + (c + 1) % L
    down = ((r + 1) % L) * L + c
    i = np.repeat(np.arange(L * L), 2)
    j = np.stack([right, down], 1).ravel()
    w = None
    if signed:
        rng = np.random.Generator(np.random.PCG64(seed))
        w = (rng.integers(0, 2, size=len(j)) * 2 - 1).astype(np.int8)
    return from_edges(L * L, i, j, w, name=f"torus{L}_s{seed}")


def delaunay(n: int, seed: int = 0) -> Graph:
    """Planar-like graph: Delaunay triangulation of n uniform points in the
    unit square (unit weights)."""
    from scipy.spatial import Delaunay

    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 2))
    tri = Delaunay(pts).simplices.astype(np.int64)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [0, 2]]])
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    return from_edges(n, e[:, 0], e[:, 1], name=f"delaunay{n}_s{seed}")


def read_gset(path: str, name: str = "") -> Graph:
    """Graph from a G-set style text file: a header line "n m", then m lines
    "i j w" with 1-based vertices and w = +1 or -1 (the benchmark format of
    the graphs named in Sec. 1)."""
    with open(path) as f:
        head = f.readline().split()
        if len(head) < 2:
            raise ValueError(f"{path}: header must be 'n m'")
        n, m = int(head[0]), int(head[1])
        rows = np.loadtxt(f, dtype=np.int64, ndmin=2) if m else np.zeros((0, 3), np.int64)
    if rows.shape != (m, 3):
        raise ValueError(f"{path}: expected {m} lines of 'i j w', found shape {rows.shape}")
    i, j, w = rows[:, 0] - 1, rows[:, 1] - 1, rows[:, 2]
    if m and (i.min() < 0 or j.min() < 0 or i.max() >= n or j.max() >= n):
        raise ValueError(f"{path}: vertex index out of 1..{n}")
    if np.any((w != 1) & (w != -1)):
        raise ValueError(f"{path}: weights must be +1 or -1")
    return from_edges(n, i, j, None if np.all(w == 1) else w.astype(np.int8),
                      name=name or os.path.basename(path))


def write_gset(g: Graph, path: str) -> None:
    """Write g in the format read_gset reads (each edge once, i < j)."""
    i, j, w = g.edges()
    with open(path, "w") as f:
        f.write(f"{g.n} {len(i)}\n")
        for a, b, c in zip(i.tolist(), j.tolist(), w.tolist()):
            f.write(f"{a + 1} {b + 1} {c}\n")


def linear_betas(lo: float, hi: float, K: int) -> np.ndarray:
    """beta_k = lo + (hi - lo) k / (K - 1), k = 0..K-1 (both ends included)."""
    if K == 1:
        return np.array([hi], np.float64)
    k = np.arange(K, dtype=np.float64)
    return lo + (hi - lo) * k / float(K - 1)


# Workloads of the evaluation (sizes of the paper's instance family; the
# anneal parameters are the ones the repository benchmarks).
CONFIGS = {
    "gnp800": dict(graph=lambda: gnp(800, 0.06, seed=0), R=256, K=100, S=4, beta=(0.1, 3.0),
                   nlm_period=0, seed=0),
    "g63like": dict(graph=lambda: gnm(7000, 41459, seed=0), R=16384, K=1000, S=10,
                    beta=(0.1, 4.0), nlm_period=50, seed=0),
    "torus100": dict(graph=lambda: torus(100, seed=0), R=32768, K=800, S=8, beta=(0.1, 3.5),
                     nlm_period=0, seed=0),
}


def batch_instances(count: int = 64, seed: int = 0):
    """Mixed batch: N ~ U[800, 20000]; kinds cycle random (p = 12/(N-1),
    M ~ 6N), signed torus (L = round(sqrt N)), Delaunay; R cycles
    1024 / 4096 / 16384."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for t in range(count):
        n = int(rng.integers(800, 20001))
        kind = t % 3
        if kind == 0:
            g = gnp_sparse(n, 12.0 / (n - 1), seed=1000 + t)
        elif kind == 1:
            g = torus(int(round(np.sqrt(n))), seed=1000 + t)
        else:
            g = delaunay(n, seed=1000 + t)
        out.append(dict(graph=g, R=(1024, 4096, 16384)[t % 3], seed=t))
    return out
