// k_moves.cu -- Houdayer non-local moves and ESS-adaptive temperature steps
// (Sec. 3 of arXiv 2510.21105 names both without defining them; the rules
// implemented here are the library's readings, stated in pa_moves.cuh).
#include <algorithm>
#include <mutex>

#include "pa_moves.cuh"

namespace pa {
namespace {

// ------------------------------------------------------------ non-local ---
// Pairing: slots sorted by (key_r, r), consecutive entries paired. The rank of
// (key_r, r) is found through NB = 2^b buckets of the top b key bits (about
// 32 slots each for uniform keys): bucket counts, their exclusive scan, the
// slots listed bucket by bucket, then each slot counts the smaller pairs of
// its own bucket. Any key distribution gives the exact rank.
struct NlmRankScratch {
    uint32_t *keys;     // [R]
    int32_t *order;     // [R] slot of each rank
    int32_t *members;   // [R] slots grouped by bucket
    int32_t *start;     // [NB + 1] bucket counts, then their exclusive scan
    int32_t *fill;      // [NB]
    int32_t NB, shift;  // bucket = NB > 1 ? key >> shift : 0
};

__host__ __device__ inline int nlm_buckets(int32_t R) {
    int nb = 1;
    while (nb < 2048 && 32 * nb < R) nb <<= 1;
    return nb;
}

__device__ __forceinline__ int nlm_bucket(uint32_t key, const NlmRankScratch &s) {
    return s.NB > 1 ? (int)(key >> s.shift) : 0;
}

__global__ void k_nlm_keys(NlmArgs a, NlmRankScratch s) {
    if (a.active && !a.active[a.k]) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r <= s.NB) s.start[r] = 0;
    if (r < s.NB) s.fill[r] = 0;
    if (r >= a.R) return;
    const uint4 u = philox10(make_uint4((uint32_t)r >> 2, 0u, (uint32_t)a.k, TAG_NONLOCAL), a.key0, a.key1);
    s.keys[r] = (r & 3) == 0 ? u.x : (r & 3) == 1 ? u.y : (r & 3) == 2 ? u.z : u.w;
}

__global__ void k_nlm_count(NlmArgs a, NlmRankScratch s) {
    if (a.active && !a.active[a.k]) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < a.R) atomicAdd(&s.start[nlm_bucket(s.keys[r], s)], 1);
}

// Exclusive scan of the NB <= 2048 bucket counts, one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_nlm_scan(NlmArgs a, NlmRankScratch s) {
    if (a.active && !a.active[a.k]) return;
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int c0 = 2 * t < s.NB ? s.start[2 * t] : 0, c1 = 2 * t + 1 < s.NB ? s.start[2 * t + 1] : 0;
    int inc = c0 + c1;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int pre = inc - c0 - c1;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    __syncthreads();   // every count is read before the starts overwrite them
    if (2 * t < s.NB) s.start[2 * t] = pre;
    if (2 * t + 1 < s.NB) s.start[2 * t + 1] = pre + c0;
    if (t == 0) s.start[s.NB] = a.R;
}

__global__ void k_nlm_fill(NlmArgs a, NlmRankScratch s) {
    if (a.active && !a.active[a.k]) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    const int b = nlm_bucket(s.keys[r], s);
    s.members[s.start[b] + atomicAdd(&s.fill[b], 1)] = r;
}

__global__ void k_nlm_rank(NlmArgs a, NlmRankScratch s) {
    if (a.active && !a.active[a.k]) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    const uint32_t kr = s.keys[r];
    const int b = nlm_bucket(kr, s);
    const int lo = s.start[b], hi = s.start[b + 1];
    int rank = lo;
    for (int i = lo; i < hi; ++i) {
        const int m = s.members[i];
        const uint32_t km = s.keys[m];
        rank += (km < kr) || (km == kr && m < r);
    }
    s.order[rank] = r;
}

// Spin bits of 32 positions (32 bytes of a row, +1 -> 1; -1 and padding -> 0).
__device__ __forceinline__ uint32_t nlm_row_bits(const int8_t *row, int w, int np) {
    uint32_t bits = 0u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p0 = 32 * w + 16 * h;
        if (p0 >= np) break;   // np is a multiple of 16
        const uint4 v = *reinterpret_cast<const uint4 *>(row + p0);
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t t = vv[q] & ~(vv[q] >> 1) & 0x01010101u;   // byte 0x01: bit 0 set, bit 1 clear
            bits |= ((t * 0x01020408u) >> 24) << (16 * h + 4 * q);
        }
    }
    return bits;
}

// One Houdayer move per pair of replicas (sa, sb), one CTA per pair. Bitsets
// over positions: Sa holds replica a's spins (+1 -> 1), D = {i : x^a_i !=
// x^b_i} (so replica b is Sa ^ D), cand = D minus the vertices already
// visited. The seed is the target-th element of D in ascending vertex order.
// A breadth-first search from it through vertices of D claims each vertex by
// clearing its cand bit (an atomic AND), so every vertex enters the queue Q
// once; Q[0, csize) is the cluster C, the seed's connected component in the
// graph induced on D. Both replicas flip on C. The visited set does not depend
// on the order in which a level is scanned.
//
// A bond (i, j) scanned from i in C leads either into D, and then j is in C
// (same component), or out of D, and then it crosses the boundary of C. So the
// search also sums the boundary bonds the energy update needs, in the same
// pass over the rows. Groups of G = 4 lanes read one vertex's row together:
// consecutive entries, fewer sectors than a lane per row, and still 64 rows
// in flight per CTA (on GB300, 4 lanes beat 1, 2 and 8 at mean degree 4 and
// 12: 2.35 and 1.05 ms per move over 16384 and 8192 pairs).
__global__ void __launch_bounds__(256) k_nlm_pair(NlmArgs a, const int32_t *order) {
    constexpr int G = 4;
    if (a.active && !a.active[a.k]) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int np = a.g.np, n = a.g.n;
    const int nw = (np + 31) >> 5;
    uint32_t *Sa = reinterpret_cast<uint32_t *>(sm);
    uint32_t *D = Sa + nw;
    uint32_t *cand = D + nw;
    uint16_t *Q = reinterpret_cast<uint16_t *>(cand + nw);   // [n] breadth-first queue
    __shared__ int sh_cnt[32];
    __shared__ int sh_nd, sh_seed, sh_tail;
    __shared__ long long sh_E[2][32];
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int gl = tid & (G - 1), grp = tid / G, NG = NT / G;
    const int m = blockIdx.x;
    const int sa = order[2 * m], sb = order[2 * m + 1];
    int8_t *ga = a.spins + (size_t)sa * np;
    int8_t *gb = a.spins + (size_t)sb * np;
    int nd_part = 0;
    for (int w = tid; w < nw; w += NT) {
        const uint32_t xa = nlm_row_bits(ga, w, np), xb = nlm_row_bits(gb, w, np);
        const int rem = n - 32 * w;   // positions of this word below n
        const uint32_t live = rem >= 32 ? 0xFFFFFFFFu : (rem <= 0 ? 0u : (1u << rem) - 1u);
        Sa[w] = xa;
        D[w] = (xa ^ xb) & live;
        cand[w] = (xa ^ xb) & live;
        nd_part += __popc((xa ^ xb) & live);
    }
    nd_part = (int)__reduce_add_sync(0xFFFFFFFFu, (uint32_t)nd_part);
    if (lane == 0) sh_cnt[warp] = nd_part;
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int w = 0; w < NT / 32; ++w) s += sh_cnt[w];
        sh_nd = s;
        sh_seed = -1;
    }
    __syncthreads();
    const int nd = sh_nd;
    if (nd == 0) return;
    // The seed: the target-th element of D in ascending vertex order. Each
    // thread counts D over a contiguous range of vertices; warp scans and the
    // warp totals give every thread its exclusive prefix.
    const uint4 u = philox10(make_uint4((uint32_t)m >> 2, 1u, (uint32_t)a.k, TAG_NONLOCAL), a.key0, a.key1);
    const uint32_t um = (m & 3) == 0 ? u.x : (m & 3) == 1 ? u.y : (m & 3) == 2 ? u.z : u.w;
    const int target = (int)(um % (uint32_t)nd);
    const int per = (n + NT - 1) / NT;
    const int i0 = tid * per, i1 = min(n, i0 + per);
    int cnt = 0;
    for (int i = i0; i < i1; ++i) {
        const int p = a.pos[i];
        cnt += (D[p >> 5] >> (p & 31)) & 1u;
    }
    int inc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) sh_cnt[warp] = inc;   // thread 0 read the counts of |D| before the last barrier
    __syncthreads();
    int pre = inc - cnt;
    for (int w = 0; w < warp; ++w) pre += sh_cnt[w];
    if (target >= pre && target < pre + cnt) {
        int c = pre;
        for (int i = i0; i < i1; ++i) {
            const int p = a.pos[i];
            if ((D[p >> 5] >> (p & 31)) & 1u) {
                if (c == target) {
                    sh_seed = p;
                    break;
                }
                ++c;
            }
        }
    }
    __syncthreads();
    if (sh_seed < 0) return;   // unreachable when nd > 0; keeps every index in range
    if (tid == 0) {
        const int s = sh_seed;
        cand[s >> 5] &= ~(1u << (s & 31));
        Q[0] = (uint16_t)s;
        sh_tail = 1;
    }
    __syncthreads();
    // Breadth-first search, one level per pass over Q[lo, hi). bnd sums
    // w_ij x^a_i x^a_j (values before the flip) over the boundary bonds.
    int lo = 0, hi = 1, bnd = 0;
    while (lo < hi) {
        for (int f = lo + grp; f < hi; f += NG) {
            const int p = Q[f];
            const uint32_t xi = (Sa[p >> 5] >> (p & 31)) & 1u;
            const uint32_t e1 = a.g.rp[p + 1];
            for (uint32_t e = a.g.rp[p] + gl; e < e1; e += G) {
                const int j = a.g.col[e];
                const uint32_t bit = 1u << (j & 31);
                if (D[j >> 5] & bit) {
                    if ((cand[j >> 5] & bit) && (atomicAnd(&cand[j >> 5], ~bit) & bit))
                        Q[atomicAdd(&sh_tail, 1)] = (uint16_t)j;
                } else {
                    const int w = a.g.wt ? (int)a.g.wt[e] : 1;
                    bnd += (((Sa[j >> 5] >> (j & 31)) & 1u) == xi) ? w : -w;
                }
            }
        }
        __syncthreads();
        lo = hi;
        hi = sh_tail;
        __syncthreads();   // every thread has read sh_tail before the next level adds to it
    }
    const int csize = hi;
    // Flip both replicas on C = D minus the remaining candidates (Sa ^ D stays
    // replica b).
    for (int w = tid; w < nw; w += NT) {
        const uint32_t c = D[w] & ~cand[w];
        if (!c) continue;
        Sa[w] ^= c;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int p0 = 32 * w + 16 * h;
            const uint32_t ch = (c >> (16 * h)) & 0xFFFFu;
            if (p0 >= np || !ch) continue;
            uint4 va = *reinterpret_cast<const uint4 *>(ga + p0), vb = *reinterpret_cast<const uint4 *>(gb + p0);
            uint32_t *pa = reinterpret_cast<uint32_t *>(&va), *pb = reinterpret_cast<uint32_t *>(&vb);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t fm = ((((ch >> (4 * q)) & 0xFu) * 0x00204081u) & 0x01010101u) * 0xFEu;   // 0x01 <-> 0xFF
                pa[q] ^= fm;
                pb[q] ^= fm;
            }
            *reinterpret_cast<uint4 *>(ga + p0) = va;
            *reinterpret_cast<uint4 *>(gb + p0) = vb;
        }
    }
    if (!a.fields) {
        // Layouts without fields: only the energies change. Flipping C in
        // both replicas exchanges their values on C, so E_a + E_b is unchanged,
        // and replica a changes by the bonds that cross the boundary of C:
        // dE_a = 2 sum_{i in C, j not in C} w_ij x'_i x'_j with the flipped
        // values x'_i = -x_i, x'_j = x_j, that is -2 bnd.
        long long d = -(long long)bnd;
        for (int off = 16; off; off >>= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, off);
        if (lane == 0) sh_E[0][warp] = d;
        __syncthreads();
        if (tid == 0) {
            long long t = 0;
            for (int w = 0; w < NT / 32; ++w) t += sh_E[0][w];
            a.E[sa] += (int32_t)(2 * t);
            a.E[sb] -= (int32_t)(2 * t);
            atomicAdd(&a.pairs[a.k], 1);
            atomicAdd(&a.flips[a.k], (unsigned long long)csize);
        }
        return;
    }
    __syncthreads();
    // Fields and energies of both replicas, recomputed.
    long long Ea = 0, Eb = 0;
    int16_t *fa = a.fields + (size_t)sa * np, *fb = a.fields + (size_t)sb * np;
    for (int base = 0; base < np; base += NG) {   // the same trip count on every lane (group shuffles)
        const int p = base + grp;
        int ha = 0, hb = 0;
        if (p < n) {
            const uint32_t e1 = a.g.rp[p + 1];
            for (uint32_t e = a.g.rp[p] + gl; e < e1; e += G) {
                const int j = a.g.col[e];
                const int w = a.g.wt ? (int)a.g.wt[e] : 1;
                const uint32_t xa = Sa[j >> 5] >> (j & 31), xb = xa ^ (D[j >> 5] >> (j & 31));
                ha += (xa & 1u) ? w : -w;
                hb += (xb & 1u) ? w : -w;
            }
        }
#pragma unroll
        for (int off = G / 2; off; off >>= 1) {
            ha += __shfl_xor_sync(0xFFFFFFFFu, ha, off);
            hb += __shfl_xor_sync(0xFFFFFFFFu, hb, off);
        }
        if (gl == 0 && p < np) {
            fa[p] = (int16_t)ha;
            fb[p] = (int16_t)hb;
            if (p < n) {
                const uint32_t xa = Sa[p >> 5] >> (p & 31), xb = xa ^ (D[p >> 5] >> (p & 31));
                Ea += (xa & 1u) ? ha : -ha;
                Eb += (xb & 1u) ? hb : -hb;
            }
        }
    }
    for (int off = 16; off; off >>= 1) {
        Ea += __shfl_xor_sync(0xFFFFFFFFu, Ea, off);
        Eb += __shfl_xor_sync(0xFFFFFFFFu, Eb, off);
    }
    if (lane == 0) {
        sh_E[0][warp] = Ea;
        sh_E[1][warp] = Eb;
    }
    __syncthreads();
    if (tid == 0) {
        long long ta = 0, tb = 0;
        for (int w = 0; w < NT / 32; ++w) {
            ta += sh_E[0][w];
            tb += sh_E[1][w];
        }
        a.E[sa] = (int32_t)(ta / 2);
        a.E[sb] = (int32_t)(tb / 2);
        atomicAdd(&a.pairs[a.k], 1);
        atomicAdd(&a.flips[a.k], (unsigned long long)csize);
    }
}

// One CTA per slot. Warp 0 grows the block by breadth-first search (lanes
// take a row's unvisited neighbours in row order through a ballot, so the
// discovery order is the sequential one); the CTA then sums the edges that
// leave the block, thread 0 decides, and an accepted move flips the block and
// rebuilds the fields of the block and its neighbours.
__global__ void __launch_bounds__(256) k_nlm_block(NlmArgs a) {
    if (a.active && !a.active[a.k]) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int np = a.g.np, n = a.g.n, nw = (np + 31) >> 5;
    int8_t *x = reinterpret_cast<int8_t *>(sm);
    uint32_t *inB = reinterpret_cast<uint32_t *>(x + np);   // np is a multiple of 16
    uint32_t *aff = inB + nw;
    int32_t *Bl = reinterpret_cast<int32_t *>(aff + nw);    // [block] positions in discovery order
    __shared__ int sh_cnt, sh_acc;
    __shared__ long long sh_red[8];
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    const int r = blockIdx.x;
    {
        const uint4 *gx = reinterpret_cast<const uint4 *>(a.spins + (size_t)r * np);
        uint4 *lx = reinterpret_cast<uint4 *>(x);
        for (int i = tid; i < (np >> 4); i += NT) lx[i] = gx[i];
        for (int i = tid; i < nw; i += NT) {
            inB[i] = 0u;
            aff[i] = 0u;
        }
    }
    __syncthreads();
    if (tid < 32) {
        const uint4 us = philox10(make_uint4((uint32_t)r >> 2, 2u, (uint32_t)a.k, TAG_NONLOCAL), a.key0, a.key1);
        const uint32_t uw[4] = {us.x, us.y, us.z, us.w};
        const int ps = a.pos[uw[r & 3] % (uint32_t)n];
        if (lane == 0) {
            Bl[0] = ps;
            inB[ps >> 5] = 1u << (ps & 31);
        }
        __syncwarp();
        int cnt = 1, head = 0;   // warp-uniform
        while (head < cnt && cnt < a.block) {
            const int p = Bl[head++];
            const uint32_t e1 = a.g.rp[p + 1];
            for (uint32_t base = a.g.rp[p]; base < e1 && cnt < a.block; base += 32) {
                const uint32_t e = base + lane;
                int j = 0;
                bool fresh = false;
                if (e < e1) {
                    j = a.g.col[e];
                    fresh = !((inB[j >> 5] >> (j & 31)) & 1u);
                }
                const uint32_t mask = __ballot_sync(0xFFFFFFFFu, fresh);
                const int take = min(__popc(mask), a.block - cnt);
                const int rank = __popc(mask & ((1u << lane) - 1u));
                if (fresh && rank < take) {
                    Bl[cnt + rank] = j;
                    atomicOr(&inB[j >> 5], 1u << (j & 31));
                }
                cnt += take;
                __syncwarp();
            }
        }
        if (lane == 0) sh_cnt = cnt;
    }
    __syncthreads();
    const int cnt = sh_cnt;
    // Sum of w x_i x_j over the edges leaving the block.
    long long lv = 0;
    for (int t = tid; t < cnt; t += NT) {
        const int p = Bl[t];
        const int xp = x[p];
        const uint32_t e1 = a.g.rp[p + 1];
        for (uint32_t e = a.g.rp[p]; e < e1; ++e) {
            const int j = a.g.col[e];
            if (!((inB[j >> 5] >> (j & 31)) & 1u)) lv += (long long)(a.g.wt ? (int)a.g.wt[e] : 1) * xp * x[j];
        }
    }
    for (int off = 16; off; off >>= 1) lv += __shfl_xor_sync(0xFFFFFFFFu, lv, off);
    if (lane == 0) sh_red[tid >> 5] = lv;
    __syncthreads();
    long long m = 0;
    for (int w = 0; w < NT / 32; ++w) m -= sh_red[w];
    if (tid == 0) {
        int acc = m <= 0;
        if (!acc) {
            const uint4 ua = philox10(make_uint4((uint32_t)r >> 2, 3u, (uint32_t)a.k, TAG_NONLOCAL), a.key0, a.key1);
            const uint32_t aw[4] = {ua.x, ua.y, ua.z, ua.w};
            double pw = 1.0, sq = a.qrow[a.tidx[a.k]];
            for (uint32_t d = (uint32_t)m; d; d >>= 1) {   // q^m: right-to-left square and multiply
                if (d & 1u) pw = __dmul_rn(pw, sq);
                sq = __dmul_rn(sq, sq);
            }
            const double v = floor(__dmul_rn(pw, 4294967296.0));
            const uint32_t A = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
            acc = aw[r & 3] < A;
        }
        sh_acc = acc;
    }
    __syncthreads();
    if (!sh_acc) return;
    int8_t *gx = a.spins + (size_t)r * np;
    for (int t = tid; t < cnt; t += NT) {
        const int p = Bl[t];
        const int8_t v = (int8_t)-x[p];
        x[p] = v;
        gx[p] = v;
        atomicOr(&aff[p >> 5], 1u << (p & 31));
        const uint32_t e1 = a.g.rp[p + 1];
        for (uint32_t e = a.g.rp[p]; e < e1; ++e) {
            const int j = a.g.col[e];
            atomicOr(&aff[j >> 5], 1u << (j & 31));
        }
    }
    __syncthreads();
    int16_t *gh = a.fields ? a.fields + (size_t)r * np : nullptr;   // null: the layout keeps no fields
    for (int p = tid; gh && p < n; p += NT)
        if ((aff[p >> 5] >> (p & 31)) & 1u) {
            int h = 0;
            const uint32_t e1 = a.g.rp[p + 1];
            for (uint32_t e = a.g.rp[p]; e < e1; ++e) h += (a.g.wt ? (int)a.g.wt[e] : 1) * x[a.g.col[e]];
            gh[p] = (int16_t)h;
        }
    if (tid == 0) {
        a.E[r] += (int32_t)(2 * m);
        atomicAdd(&a.pairs[a.k], 1);
        atomicAdd(&a.flips[a.k], (unsigned long long)cnt);
    }
}

// -------------------------------------------------------------- adaptive ---
// ESS partials, one CTA per (256-slot chunk, level j): w = q_j^(E - E_min) by
// squarings and w*w for one slot per thread, then the chunk's pairwise tree
// sums (lanes by butterflies, then the eight warp sums in pairs), the same
// additions as the tree over the whole padded population.
__global__ void __launch_bounds__(RS_CHUNK) k_ad_partials(AdaptArgs a) {
    const int n_prev = a.state[0];
    if (n_prev >= a.nmax) return;
    __shared__ double sw[2][RS_CHUNK / 32];
    const int j = blockIdx.y;
    const int slot = blockIdx.x * RS_CHUNK + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int dn = 1 << (a.J - j);
    if (dn > a.nmax - n_prev) dn = a.nmax - n_prev;
    const double *qs = a.qpow + (size_t)(dn - 1) * 32;
    double w = 0.0;
    if (slot < a.R) {
        w = 1.0;
        uint32_t dd = (uint32_t)(a.E[slot] - a.emin[a.k]);
        while (dd) {
            w = __dmul_rn(w, __ldg(&qs[__ffs(dd) - 1]));
            dd &= dd - 1u;
        }
    }
    double s = w, s2 = __dmul_rn(w, w);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        s = __dadd_rn(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
        s2 = __dadd_rn(s2, __shfl_xor_sync(0xFFFFFFFFu, s2, off));
    }
    if (lane == 0) {
        sw[0][warp] = s;
        sw[1][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double *v = sw[threadIdx.x];
        for (int h = 1; h < RS_CHUNK / 32; h <<= 1)
            for (int i = 0; i < RS_CHUNK / 32; i += 2 * h) v[i] = __dadd_rn(v[i], v[i + h]);
        a.part[((size_t)j * 2 + threadIdx.x) * a.nch + blockIdx.x] = v[0];
    }
}

// Pairwise tree sum of v[0..n) padded with zeros to a power of two, computed
// left to right with a stack of completed subtrees (same additions as the
// level-by-level tree).
__device__ double tree_sum_seq(const double *v, int n) {
    double st[20];
    int lv[20];
    int top = 0;
    int L = 1;
    while (L < n) L <<= 1;
    for (int i = 0; i < L; ++i) {
        double x = i < n ? v[i] : 0.0;
        int l = 0;
        while (top > 0 && lv[top - 1] == l) {
            x = __dadd_rn(st[top - 1], x);
            --top;
            ++l;
        }
        st[top] = x;
        lv[top] = l;
        ++top;
    }
    return st[0];
}

// Level choice. Mode 1: one warp per level j sums the chunk partials of w and
// w*w in the tree's order (each lane a contiguous power-of-two block of
// chunks, then butterflies; zero padding adds exact zeros), ESS_j = A^2 / B,
// and the smallest j with ESS_j >= rho R is taken (else J).
__global__ void k_ad_choose(AdaptArgs a) {
    const int n_prev = a.state[0];
    const int lane = threadIdx.x & 31, lvl = threadIdx.x >> 5;
    __shared__ int ok_lvl[32];
    if (n_prev >= a.nmax) {
        if (threadIdx.x == 0) a.active[a.k] = 0;
        return;
    }
    if (a.mode == 2) {
        if (threadIdx.x == 0) {
            int j = a.state[1];
            if (a.k > 0) {
                const double acc = (double)a.accepts[a.k - 1];
                if (acc < a.acc_lo_n) j = min(j + 1, a.J);
                else if (acc > a.acc_hi_n) j = max(j - 1, 0);
            }
            int dn = 1 << (a.J - j);
            if (dn > a.nmax - n_prev) dn = a.nmax - n_prev;
            const int nk = n_prev + dn;
            a.state[0] = nk;
            a.state[1] = j;
            a.qsel[a.k] = dn - 1;
            a.tidx[a.k] = nk;
            a.jsel[a.k] = j;
            a.beta[a.k] = __dmul_rn((double)nk, a.delta);
            a.active[a.k] = 1;
        }
        return;
    }
    if (lvl <= a.J) {
        int L = 1;
        while (L < a.nch) L <<= 1;
        const int blk = L > 32 ? L / 32 : 1;
        const int lo = lane * blk, cnt = max(0, min(blk, a.nch - lo));
        double A = tree_sum_seq(a.part + ((size_t)lvl * 2 + 0) * a.nch + min(lo, a.nch), cnt);
        double B = tree_sum_seq(a.part + ((size_t)lvl * 2 + 1) * a.nch + min(lo, a.nch), cnt);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            A = __dadd_rn(A, __shfl_xor_sync(0xFFFFFFFFu, A, off));
            B = __dadd_rn(B, __shfl_xor_sync(0xFFFFFFFFu, B, off));
        }
        if (lane == 0) ok_lvl[lvl] = __ddiv_rn(__dmul_rn(A, A), B) >= a.rhoR;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int j = a.J;
        for (int l = 0; l < a.J; ++l)
            if (ok_lvl[l]) {
                j = l;
                break;
            }
        int dn = 1 << (a.J - j);
        if (dn > a.nmax - n_prev) dn = a.nmax - n_prev;
        const int nk = n_prev + dn;
        a.state[0] = nk;
        a.qsel[a.k] = dn - 1;
        a.tidx[a.k] = nk;
        a.jsel[a.k] = j;
        a.beta[a.k] = __dmul_rn((double)nk, a.delta);
        a.active[a.k] = 1;
    }
}

// ------------------------------------------------------------- reheating ---
__global__ void k_rh_choose(ReheatArgs a) {
    if (threadIdx.x != 0) return;
    int i = 0, row = 0;
    if (a.k > 0) {
        const int ip = a.state[0];
        int stall = a.state[1], best = a.state[2];
        int step_min = 0x7FFFFFFF;
        for (int s = 0; s < a.S; ++s) step_min = min(step_min, a.sweep_emin[(size_t)(a.k - 1) * a.S + s]);
        if (step_min < best) {
            best = step_min;
            stall = 0;
        } else {
            ++stall;
        }
        if (stall >= a.after) {
            i = max(0, ip - a.back);
            stall = 0;
        } else {
            i = min(ip + 1, a.K - 1);
        }
        row = i == ip + 1 ? i : a.K;
        a.state[1] = stall;
        a.state[2] = best;
    } else {
        a.state[1] = 0;
        a.state[2] = 0x7FFFFFFF;
    }
    a.state[0] = i;
    a.tidx[a.k] = i;
    a.qsel[a.k] = row;
    a.isel[a.k] = i;
    a.beta[a.k] = a.betas[i];
}

}  // namespace

cudaError_t launch_reheat(const ReheatArgs &a, cudaStream_t st) {
    k_rh_choose<<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

size_t nlm_scratch_bytes(int32_t R) {   // keys, order, members, bucket starts and fills
    return (size_t)R * 12 + (size_t)(2 * nlm_buckets(R) + 1) * 4 + 256;
}

size_t nlm_smem_bytes(int32_t np) {   // spin bitsets of both replicas, candidates, queue
    return 3 * 4 * (size_t)((np + 31) / 32) + 2 * (size_t)np + 16;
}

size_t nlm_block_smem_bytes(int32_t np, int32_t block) {
    return (size_t)np + 8 * (size_t)((np + 31) / 32) + 4 * (size_t)block;
}

cudaError_t launch_nonlocal(const NlmArgs &a, void *scratch, cudaStream_t st, int *launches) {
    if (a.kind == 1) {
        *launches = 0;
        if (a.R < 1) return cudaSuccess;
        const size_t smem = nlm_block_smem_bytes(a.g.np, a.block);
        static std::mutex mu;
        static size_t raised = 48 * 1024;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (smem > raised) {   // per-function attribute: only ever raise it
                cudaError_t e = cudaFuncSetAttribute(k_nlm_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                raised = smem;
            }
        }
        // Two warps per slot: the search is one warp's work, so small CTAs keep
        // more searches in flight per SM.
        k_nlm_block<<<a.R, 64, smem, st>>>(a);
        *launches = 1;
        return cudaGetLastError();
    }
    NlmRankScratch rs;
    rs.keys = reinterpret_cast<uint32_t *>(scratch);
    rs.order = reinterpret_cast<int32_t *>(rs.keys + a.R);
    rs.members = rs.order + a.R;
    rs.NB = nlm_buckets(a.R);
    rs.start = rs.members + a.R;
    rs.fill = rs.start + rs.NB + 1;
    int lg = 0;
    while ((1 << lg) < rs.NB) ++lg;
    rs.shift = 32 - lg;
    const int nb = (a.R + 255) / 256;
    k_nlm_keys<<<(std::max(a.R, rs.NB + 1) + 255) / 256, 256, 0, st>>>(a, rs);
    k_nlm_count<<<nb, 256, 0, st>>>(a, rs);
    k_nlm_scan<<<1, 1024, 0, st>>>(a, rs);
    k_nlm_fill<<<nb, 256, 0, st>>>(a, rs);
    k_nlm_rank<<<nb, 256, 0, st>>>(a, rs);
    const int32_t *order = rs.order;
    *launches = 5;
    if (a.R >= 2) {
        const size_t smem = nlm_smem_bytes(a.g.np);
        static std::mutex mu;
        static size_t raised = 0;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (smem > raised) {   // per-function attribute: only ever raise it
                cudaError_t e = cudaFuncSetAttribute(k_nlm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                raised = smem;
            }
        }
        k_nlm_pair<<<a.R / 2, 256, smem, st>>>(a, order);
        *launches = 6;
    }
    return cudaGetLastError();
}

cudaError_t launch_adapt(const AdaptArgs &a, cudaStream_t st) {
    if (a.mode != 2) k_ad_partials<<<dim3(a.nch, a.J + 1), RS_CHUNK, 0, st>>>(a);
    k_ad_choose<<<1, a.mode == 2 ? 32 : 32 * (a.J + 1), 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace pa
