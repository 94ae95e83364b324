// k_resample.cu -- population initialisation, local fields / energies, and the
// per-temperature-step reweighting + resampling of PAMC (Sec. 3 of arXiv
// 2510.21105 names population annealing; the scheme below is the library's
// reading of it).
//
// Resampling of step k (energies E_r of the R replicas entering the step):
//   E_min = min_r E_r, d_r = E_r - E_min
//   w_r   = q^{d_r}, q = exp(-(beta_k - beta_{k-1})), as the product of the
//           host-computed squarings q^(2^b) over the set bits b of d_r in
//           ascending b (FP64, round to nearest, no fused operations)
//   A     = sum of w_r as a pairwise tree over slots padded to a power of two
//   t_r   = floor(2^32 w_r) (integer weights), T = sum t_r, P_r = sum_{s<r} t_s
//   new slots [F(P_r), F(P_r + t_r)) copy replica r, with the systematic
//   count F(P) = floor((P R 2^32 + o T) / (T 2^32)) and o the Philox word of
//   (0, 0, k, tag 1). Sum of copies is exactly R.
// Three kernels per step over chunks of RS_CHUNK slots: minimum, weights
// (chunk tree sums of w, chunk totals and local prefixes of t), parents.
#include "pa_internal.cuh"

namespace pa {
namespace {

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_init_spins(GraphDev g, int8_t *spins, int32_t Rpad, uint32_t k0, uint32_t k1) {
    const int nchunk = g.np >> 2;
    const long total = (long)(Rpad >> 2) * nchunk;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int grp = (int)(idx / nchunk), c = (int)(idx % nchunk);
        uint32_t out[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = 4 * c + j;
            if (p < g.n) {
                const uint4 u = philox10(make_uint4(g.vid[p], (uint32_t)grp, 0u, TAG_INIT), k0, k1);
                const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) out[q] |= ((uu[q] >> 31) ? 0x01u : 0xFFu) << (8 * j);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint32_t *>(spins + (size_t)(4 * grp + q) * g.np + 4 * c) = out[q];
    }
}

// One CTA per replica: h_p = sum_j w_pj x_j and E = 1/2 sum_p x_p h_p.
__global__ void k_fields_energy(GraphDev g, const int8_t *spins, int16_t *fields, int32_t *E) {
    const int r = blockIdx.x;
    const int8_t *x = spins + (size_t)r * g.np;
    int16_t *h = fields + (size_t)r * g.np;
    long long acc = 0;
    for (int p = threadIdx.x; p < g.np; p += blockDim.x) {
        int hp = 0;
        if (p < g.n) {
            const uint32_t e1 = g.rp[p + 1];
            for (uint32_t e = g.rp[p]; e < e1; ++e) {
                const int xj = x[g.col[e]];
                hp += g.wt ? (int)g.wt[e] * xj : xj;
            }
            acc += (long long)x[p] * hp;
        }
        h[p] = (int16_t)hp;
    }
    __shared__ long long red[32];
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        E[r] = (int32_t)(t / 2);
    }
}

// The resampling kernels run one CTA of RS_CHUNK threads per chunk of
// RS_CHUNK slots, one slot per thread.
__global__ void __launch_bounds__(RS_CHUNK) k_rs_min(ResampleArgs a) {
    if (a.active && !a.active[a.k]) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.stamp[a.k] = gtimer();
    const int r = blockIdx.x * RS_CHUNK + threadIdx.x;
    int v = r < a.R ? a.E[r] : 0x7FFFFFFF;
    v = __reduce_min_sync(0xFFFFFFFFu, v);
    if ((threadIdx.x & 31) == 0) atomicMin(&a.emin[a.k], v);
}

__global__ void __launch_bounds__(RS_CHUNK) k_rs_weights(ResampleArgs a) {
    if (a.active && !a.active[a.k]) return;
    __shared__ double qs[32];
    __shared__ double wsum[RS_CHUNK / 32];
    __shared__ unsigned long long tsum[RS_CHUNK / 32];
    const int row = a.qsel ? a.qsel[a.k] : a.k;
    if (threadIdx.x < 32) qs[threadIdx.x] = a.qpow[(size_t)row * 32 + threadIdx.x];
    __syncthreads();
    const int r = blockIdx.x * RS_CHUNK + threadIdx.x;
    double w = 0.0;
    unsigned long long t = 0ull;
    if (r < a.R) {
        uint32_t d = (uint32_t)(a.E[r] - a.emin[a.k]);
        w = 1.0;
        while (d) {
            w = __dmul_rn(w, qs[__ffs(d) - 1]);
            d &= d - 1u;
        }
        t = (unsigned long long)__dmul_rn(w, 4294967296.0);
    }
    // Pairwise tree: lane butterflies (32 slots), then the eight warp sums in pairs.
    double s = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) s = __dadd_rn(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
    // Exclusive prefix of t over the chunk.
    unsigned long long inc = t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) {
        wsum[warp] = s;
        tsum[warp] = inc;
    }
    __syncthreads();
    unsigned long long pre = inc - t;
    for (int w2 = 0; w2 < warp; ++w2) pre += tsum[w2];
    a.ploc[r] = pre;   // sized nch * RS_CHUNK; slots past R hold t = 0
    a.tval[r] = t;
    if (threadIdx.x == 0) {
        for (int h = 1; h < RS_CHUNK / 32; h <<= 1)
            for (int i = 0; i < RS_CHUNK / 32; i += 2 * h) wsum[i] = __dadd_rn(wsum[i], wsum[i + h]);
        unsigned long long ct = 0;
        for (int w2 = 0; w2 < RS_CHUNK / 32; ++w2) ct += tsum[w2];
        a.partA[blockIdx.x] = wsum[0];
        a.partT[blockIdx.x] = ct;
    }
}

// floor((P R 2^32 + o T) / (T 2^32)) for R <= 65536, written as
// floor(P R / T) + [ (P R mod T) 2^32 >= T (2^32 - o) ]. The division by T
// goes through m = floor((2^64 - 1) / T), computed once per step: q =
// mulhi(X, m) satisfies X/T - 2 < q <= X/T (m >= (2^64 - T)/T and X < 2^64),
// so at most two corrections make it exact.
__device__ __forceinline__ int32_t systematic_count_m(unsigned long long P, int32_t R, unsigned long long T,
                                                      unsigned long long m, uint32_t o) {
    if (P >= T) return R;
    const unsigned long long X = P * (unsigned long long)R;
    unsigned long long q = __umul64hi(X, m), r = X - q * T;
    if (r >= T) {
        ++q;
        r -= T;
    }
    if (r >= T) {
        ++q;
        r -= T;
    }
    const unsigned __int128 lhs = (unsigned __int128)r << 32;
    const unsigned __int128 rhs = (unsigned __int128)T * (0x100000000ull - (unsigned long long)o);
    return (int32_t)(q + (lhs >= rhs ? 1ull : 0ull));
}

__global__ void __launch_bounds__(RS_CHUNK) k_rs_parents(ResampleArgs a) {
    if (a.active && !a.active[a.k]) return;
    __shared__ unsigned long long sh_T, sh_off, sh_m;
    __shared__ uint32_t sh_o;
    if (threadIdx.x < 32) {   // warp 0: totals over the chunks
        const int lane = threadIdx.x;
        // T and this chunk's offset: integer sums, in any order.
        unsigned long long T = 0, off = 0;
        for (int c = lane; c < a.nch; c += 32) {
            const unsigned long long t = a.partT[c];
            T += t;
            off += c < (int)blockIdx.x ? t : 0ull;
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T += __shfl_xor_sync(0xFFFFFFFFu, T, d);
            off += __shfl_xor_sync(0xFFFFFFFFu, off, d);
        }
        // A: the pairwise tree over the chunk sums padded with zeros to a power
        // of two L <= 256. Lane l holds the aligned block of B = max(L/32, 1)
        // chunks starting at l B: the tree levels inside the block run in the
        // lane, the remaining levels pair lanes l and l ^ d, so every level adds
        // elements 2i and 2i + 1 of the level below, as the sequential tree does.
        double A = 0.0;
        if (blockIdx.x == 0) {
            int L = 1;
            while (L < a.nch) L <<= 1;
            const int B = L > 32 ? L / 32 : 1;
            double v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = lane * B + j;
                v[j] = (j < B && c < a.nch) ? a.partA[c] : 0.0;
            }
#pragma unroll
            for (int w = 1; w < 8; w <<= 1)
#pragma unroll
                for (int j = 0; j < 8; j += 2 * w)
                    if (w < B) v[j] = __dadd_rn(v[j], v[j + w]);
            A = v[0];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) A = __dadd_rn(A, __shfl_xor_sync(0xFFFFFFFFu, A, d));
        }
        if (lane == 0) {
            sh_T = T;
            sh_m = T ? ~0ull / T : 0ull;
            sh_off = off;
            sh_o = philox10(make_uint4(0u, 0u, (uint32_t)a.k, TAG_RESAMPLE), a.key0, a.key1).x;
            if (blockIdx.x == 0) {
                a.recA[a.k] = A;
                a.recT[a.k] = T;
                a.reco[a.k] = sh_o;
            }
        }
    }
    __syncthreads();
    const unsigned long long T = sh_T, off = sh_off, m = sh_m;
    const uint32_t o = sh_o;
    const int r = blockIdx.x * RS_CHUNK + threadIdx.x;
    // Slot r fills new slots [F(P_r), F(P_r + t_r)); P_r + t_r = P_{r+1} inside
    // the chunk, so the upper end is the next lane's lower end.
    const unsigned long long P = off + a.ploc[r];
    const int32_t lo = systematic_count_m(P, a.R, T, m, o);
    int32_t hi = __shfl_down_sync(0xFFFFFFFFu, lo, 1);
    if ((threadIdx.x & 31) == 31) hi = systematic_count_m(P + a.tval[r], a.R, T, m, o);
    if (r < a.R) {
        for (int s = lo; s < hi; ++s) a.parent[s] = r;
        if (a.counts) a.counts[(size_t)a.k * a.R + r] = hi - lo;
    }
}

__global__ void k_stamp(unsigned long long *stamp) { *stamp = gtimer(); }

}  // namespace

cudaError_t launch_init(const GraphDev &g, int8_t *spins, int32_t Rpad, uint32_t key0,
                        uint32_t key1, cudaStream_t st) {
    const long total = (long)(Rpad >> 2) * (g.np >> 2);
    long blocks = (total + 255) / 256;
    if (blocks > 65535L * 16) blocks = 65535L * 16;
    k_init_spins<<<(unsigned)blocks, 256, 0, st>>>(g, spins, Rpad, key0, key1);
    return cudaGetLastError();
}

cudaError_t launch_fields(const GraphDev &g, const int8_t *spins, int16_t *fields, int32_t *E,
                          int32_t Rpad, cudaStream_t st) {
    k_fields_energy<<<Rpad, 256, 0, st>>>(g, spins, fields, E);
    return cudaGetLastError();
}

cudaError_t launch_rs_min(const ResampleArgs &a, cudaStream_t st) {
    k_rs_min<<<a.nch, RS_CHUNK, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rs_rest(const ResampleArgs &a, cudaStream_t st) {
    k_rs_weights<<<a.nch, RS_CHUNK, 0, st>>>(a);
    k_rs_parents<<<a.nch, RS_CHUNK, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stamp(unsigned long long *stamp, cudaStream_t st) {
    k_stamp<<<1, 1, 0, st>>>(stamp);
    return cudaGetLastError();
}

}  // namespace pa
