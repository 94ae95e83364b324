// pa_shard.cu -- resampling of one population split over G ranks (replica
// sharding). Each rank holds the aligned power-of-two slot range
// [g R/G, (g+1) R/G) of a population of R = 2^a replicas, so its slots form
// one subtree of the pairwise weight tree of the single-population resampling
// (Sec. 3 names population annealing; the reweighting and systematic
// resampling follow the library's reading: weights q^(E - E_min) as FP64
// products of squarings, pairwise tree sum A, integer weights floor(2^32 w),
// copies F(P + t) - F(P) with F(P) = floor((P R 2^32 + o T) / (T 2^32))).
//
// One step on rank g:
//   1. pa_shard_min       E_min,g of the rank's energies; the caller reduces
//                         E_min = min over ranks;
//   2. pa_shard_partials  weights with that E_min, the subtree sum A_g, the
//                         integer weights t_r, their total T_g and local
//                         exclusive prefix, in caller scratch;
//   3. the caller gathers (A_h, T_h) of every rank;
//   4. pa_shard_plan      (host) A = pairwise tree over the A_h in rank order,
//                         which is the top of the single-population tree, so A
//                         is bitwise the single-population value; T = sum T_h;
//                         P_base = sum_{h<g} T_h; the new slots this rank's
//                         parents fill, [F(P_base), F(P_base + T_g)) (systematic
//                         resampling keeps parent order, so they are contiguous),
//                         and how many rows go to and come from every rank;
//   5. pa_shard_parents   for each of those new slots, its local parent;
//   6. pa_shard_gather    the rows (spins, energy) in new-slot order, ready
//                         for an all-to-all whose send counts pa_shard_plan
//                         gave; received rows arrive in new-slot order.
// All integer sums are exact, so counts, parents and rows equal the
// single-population resampling bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace {

constexpr int SH_THREADS = 1024;

struct QPow {
    double v[32];   // squarings of q = exp(-(beta_k - beta_prev))
};

__global__ void __launch_bounds__(SH_THREADS) k_shard_min(const int32_t *__restrict__ E, int32_t n,
                                                          int32_t *__restrict__ out) {
    __shared__ int32_t sh[SH_THREADS / 32];
    int v = 0x7FFFFFFF;
    for (int r = threadIdx.x; r < n; r += SH_THREADS) v = min(v, E[r]);
    v = __reduce_min_sync(0xFFFFFFFFu, v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = sh[0];
        for (int w = 1; w < SH_THREADS / 32; ++w) m = min(m, sh[w]);
        *out = m;
    }
}

// Scratch (caller device memory, pa_shard_scratch_bytes(n)): w[L], w2[L/2]
// doubles for the tree (L = n rounded up to a power of two), t[n] and pre[n]
// (exclusive prefix) as 64-bit integers, then A and T.
struct ShardScratch {
    double *w, *w2;
    unsigned long long *t, *pre;
    double *A;
    unsigned long long *T;
};

__host__ __device__ inline int32_t pow2_ceil(int32_t n) {
    int32_t L = 1;
    while (L < n) L <<= 1;
    return L;
}

__host__ __device__ inline ShardScratch scratch_view(void *base, int32_t n) {
    const int32_t L = pow2_ceil(n);
    ShardScratch s;
    s.w = reinterpret_cast<double *>(base);
    s.w2 = s.w + L;
    s.t = reinterpret_cast<unsigned long long *>(s.w2 + (L > 1 ? L / 2 : 1));
    s.pre = s.t + n;
    s.A = reinterpret_cast<double *>(s.pre + n);
    s.T = reinterpret_cast<unsigned long long *>(s.A + 1);
    return s;
}

__global__ void __launch_bounds__(SH_THREADS) k_shard_partials(const int32_t *__restrict__ E, int32_t n,
                                                               int32_t emin, const QPow qp, ShardScratch s) {
    __shared__ unsigned long long sh_u[SH_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = pow2_ceil(n);
    for (int r = tid; r < L; r += SH_THREADS) {
        double acc = 0.0;
        if (r < n) {
            acc = 1.0;
            uint32_t d = (uint32_t)(E[r] - emin);
            while (d) {
                const int b = __ffs(d) - 1;
                acc = __dmul_rn(acc, qp.v[b]);
                d &= d - 1u;
            }
            s.t[r] = (unsigned long long)__dmul_rn(acc, 4294967296.0);
        }
        s.w[r] = acc;
    }
    __syncthreads();
    // Pairwise tree over the slots padded with zeros to L: s_i <- s_2i + s_2i+1.
    double *src = s.w, *dst = s.w2;
    for (int len = L; len > 1; len >>= 1) {
        for (int i = tid; i < len / 2; i += SH_THREADS) dst[i] = __dadd_rn(src[2 * i], src[2 * i + 1]);
        __syncthreads();
        double *tmp = src;
        src = dst;
        dst = tmp;
    }
    // Exclusive prefix of t: contiguous chunks per thread, then across threads.
    const int chunk = (n + SH_THREADS - 1) / SH_THREADS;
    const int r0 = tid * chunk, r1 = min(n, r0 + chunk);
    unsigned long long loc = 0ull;
    for (int r = r0; r < r1; ++r) loc += s.t[r];
    unsigned long long inc = loc;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) sh_u[warp] = inc;
    __syncthreads();
    unsigned long long pre = inc - loc;
    for (int w = 0; w < warp; ++w) pre += sh_u[w];
    for (int r = r0; r < r1; ++r) {
        s.pre[r] = pre;
        pre += s.t[r];
    }
    if (tid == 0) {
        unsigned long long T = 0ull;
        for (int w = 0; w < SH_THREADS / 32; ++w) T += sh_u[w];
        *s.A = src[0];
        *s.T = T;
    }
}

// floor((P R 2^32 + o T) / (T 2^32)) for R <= 65536 (P R < 2^64): written as
// floor(P R / T) + [(P R mod T) 2^32 >= T (2^32 - o)].
__host__ __device__ inline int32_t shard_count(unsigned long long P, int32_t R, unsigned long long T, uint32_t o) {
    if (P >= T) return R;
    const unsigned long long X = P * (unsigned long long)R;
    const unsigned long long q = X / T, r = X - q * T;
    const unsigned __int128 lhs = (unsigned __int128)r << 32;
    const unsigned __int128 rhs = (unsigned __int128)T * (0x100000000ull - (unsigned long long)o);
    return (int32_t)(q + (lhs >= rhs ? 1ull : 0ull));
}

__global__ void k_shard_parents(ShardScratch s, int32_t n, unsigned long long P_base, unsigned long long T,
                                int32_t R, uint32_t o, int32_t new_lo, int32_t *__restrict__ src,
                                int32_t *__restrict__ counts) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const unsigned long long P = P_base + s.pre[r];
        const int32_t lo = shard_count(P, R, T, o), hi = shard_count(P + s.t[r], R, T, o);
        for (int32_t q = lo; q < hi; ++q) src[q - new_lo] = r;
        if (counts) counts[r] = hi - lo;
    }
}

__global__ void k_shard_gather(const int8_t *__restrict__ spins, const int32_t *__restrict__ E, int32_t ncols,
                               const int32_t *__restrict__ src, int32_t nout, int8_t *__restrict__ spins_out,
                               int32_t *__restrict__ E_out) {
    for (int j = blockIdx.x; j < nout; j += gridDim.x) {
        const int32_t r = src[j];
        const int8_t *in = spins + (size_t)r * ncols;
        int8_t *out = spins_out + (size_t)j * ncols;
        for (int c = threadIdx.x; c < ncols; c += blockDim.x) out[c] = in[c];
        if (threadIdx.x == 0 && E) E_out[j] = E[r];
    }
}

bool is_pow2(int32_t x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

extern "C" {

size_t pa_shard_scratch_bytes(int32_t n) {
    if (n < 1) return 0;
    const size_t L = (size_t)pow2_ceil(n);
    return 8 * (L + (L > 1 ? L / 2 : 1) + 2 * (size_t)n + 2);
}

int pa_shard_min(const int32_t *energies, int32_t n, int32_t *scratch, int32_t *emin, void *stream) {
    if (!energies || !scratch || !emin || n < 1) return PA_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_shard_min<<<1, SH_THREADS, 0, st>>>(energies, n, scratch);
    if (cudaGetLastError() != cudaSuccess) return PA_ECUDA;
    if (cudaMemcpyAsync(emin, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PA_ECUDA;
    return PA_OK;
}

int pa_shard_partials(const int32_t *energies, int32_t n, int32_t emin, double beta_prev, double beta_k,
                      void *scratch, double *A, uint64_t *T, void *stream) {
    if (!energies || !scratch || !A || !T || n < 1 || n > PA_SHARD_MAX_SLOTS) return PA_EINVAL;
    if (!std::isfinite(beta_prev) || !std::isfinite(beta_k) || beta_prev < 0.0 || beta_k < beta_prev) return PA_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    QPow qp;
    double sq = std::exp(-(beta_k - beta_prev));
    for (int b = 0; b < 32; ++b) {
        qp.v[b] = sq;
        sq = sq * sq;
    }
    const ShardScratch s = scratch_view(scratch, n);
    k_shard_partials<<<1, SH_THREADS, 0, st>>>(energies, n, emin, qp, s);
    if (cudaGetLastError() != cudaSuccess) return PA_ECUDA;
    unsigned long long Tv = 0;
    if (cudaMemcpyAsync(A, s.A, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&Tv, s.T, sizeof(Tv), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PA_ECUDA;
    *T = Tv;
    return PA_OK;
}

int pa_shard_plan(int32_t G, int32_t g, int32_t R, const double *A_all, const uint64_t *T_all, uint32_t o,
                  pa_shard_step *out) {
    if (!A_all || !T_all || !out || !is_pow2(G) || G > PA_SHARD_MAX_RANKS || g < 0 || g >= G || !is_pow2(R) ||
        R > 65536 || R < G)
        return PA_EINVAL;
    // Top of the pairwise tree: rank subtrees combined in rank order.
    double lvl[PA_SHARD_MAX_RANKS];
    for (int h = 0; h < G; ++h) lvl[h] = A_all[h];
    for (int len = G; len > 1; len >>= 1)
        for (int i = 0; i < len / 2; ++i) lvl[i] = lvl[2 * i] + lvl[2 * i + 1];
    unsigned long long T = 0, base[PA_SHARD_MAX_RANKS + 1];
    for (int h = 0; h < G; ++h) {
        base[h] = T;
        T += T_all[h];
    }
    base[G] = T;
    if (T == 0) return PA_EINVAL;   // every weight underflowed: impossible with E_min from the data
    const int32_t width = R / G;
    out->A = lvl[0];
    out->T = T;
    out->P_base = base[g];
    out->new_lo = shard_count(base[g], R, T, o);
    out->new_hi = shard_count(base[g + 1], R, T, o);
    for (int h = 0; h < PA_SHARD_MAX_RANKS; ++h) out->send[h] = out->recv[h] = 0;
    for (int h = 0; h < G; ++h) {
        // rows this rank sends to rank h, and rows rank h's parents send here
        const int32_t lo = h * width, hi = lo + width;
        out->send[h] = (int32_t)std::max(0, std::min(out->new_hi, hi) - std::max(out->new_lo, lo));
        const int32_t hlo = shard_count(base[h], R, T, o), hhi = shard_count(base[h + 1], R, T, o);
        out->recv[h] = (int32_t)std::max(0, std::min(hhi, g * width + width) - std::max(hlo, g * width));
    }
    return PA_OK;
}

int pa_shard_parents(const void *scratch, int32_t n, int32_t R, uint32_t o, const pa_shard_step *step,
                     int32_t *src, int32_t *counts, void *stream) {
    if (!scratch || !step || (!src && step->new_hi > step->new_lo) || n < 1 || n > PA_SHARD_MAX_SLOTS || R < 1 || R > 65536) return PA_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const ShardScratch s = scratch_view(const_cast<void *>(scratch), n);
    k_shard_parents<<<(n + 255) / 256, 256, 0, st>>>(s, n, step->P_base, step->T, R, o, step->new_lo, src, counts);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ECUDA;
}

int pa_shard_gather(const int8_t *spins, const int32_t *energies, int32_t ncols, const int32_t *src, int32_t nout,
                    int8_t *spins_out, int32_t *energies_out, void *stream) {
    if (nout == 0) return PA_OK;   // a rank whose parents fill no new slot sends nothing
    if (!spins || !src || !spins_out || ncols < 1 || nout < 0 || (energies && !energies_out)) return PA_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int grid = nout < 4096 ? nout : 4096;
    k_shard_gather<<<grid, 128, 0, st>>>(spins, energies, ncols, src, nout, spins_out, energies_out);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ECUDA;
}

uint32_t pa_resample_offset(uint64_t seed, int32_t k) {
    return pa::philox10(make_uint4(0u, 0u, (uint32_t)k, pa::TAG_RESAMPLE), (uint32_t)seed, (uint32_t)(seed >> 32)).x;
}

}  // extern "C"
