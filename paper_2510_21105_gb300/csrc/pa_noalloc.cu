// pa_noalloc.cu -- pa_resample_noalloc(): one resampling step that allocates
// no memory. For callers that cannot call cudaMalloc: a host framework that
// owns the device-memory budget through its own pool, and latency-critical
// loops where an allocator call may block, synchronise or fail. The caller
// passes the energies and receives the parents and copy counts in its own
// device buffers; every intermediate array lives in one file-scope __device__
// scratch buffer of fixed size, shared by all calls.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace {

constexpr int NA_MAX_R = PA_NOALLOC_MAX_R;   // 32768 replicas
constexpr int NA_THREADS = 1024;

struct QPow {
    double v[32];                      // squarings of q = exp(-(beta_k - beta_prev))
};

struct NoallocScratch {
    double w[NA_MAX_R];                // weights, then the tree levels (ping)
    double w2[NA_MAX_R / 2];           // tree levels (pong)
    unsigned long long t[NA_MAX_R];    // integer weights floor(2^32 w)
    double A;
    unsigned long long T;
    int32_t emin;
    uint32_t o;
};

// Every GPU that loads the library holds this buffer (about 0.6 MB) until the
// process exits. Each call writes every field it reads before reading it, so
// the previous call's contents never need clearing.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

__device__ __forceinline__ int32_t na_count(unsigned long long P, int32_t R, unsigned long long T, uint32_t o) {
    if (P >= T) return R;
    const unsigned long long X = P * (unsigned long long)R;
    const unsigned long long q = X / T, r = X - q * T;
    const unsigned __int128 lhs = (unsigned __int128)r << 32;
    const unsigned __int128 rhs = (unsigned __int128)T * (0x100000000ull - (unsigned long long)o);
    return (int32_t)(q + (lhs >= rhs ? 1ull : 0ull));
}

// One CTA: minimum, weights, pairwise tree sum, prefix of the integer
// weights, systematic copy counts and parents (same arithmetic as the
// resampling inside pa_anneal).
__global__ void __launch_bounds__(NA_THREADS) k_resample_noalloc(const int32_t *__restrict__ E, int32_t R,
                                                                 NoallocScratch *s, const QPow qp, uint32_t key0,
                                                                 uint32_t key1, uint32_t k,
                                                                 int32_t *__restrict__ parent,
                                                                 int32_t *__restrict__ counts) {
    __shared__ int32_t sh_i[32];
    __shared__ unsigned long long sh_u[32];
    __shared__ int32_t sh_emin;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int v = 0x7FFFFFFF;
    for (int r = tid; r < R; r += NA_THREADS) v = min(v, E[r]);
    v = __reduce_min_sync(0xFFFFFFFFu, v);
    if (lane == 0) sh_i[warp] = v;
    __syncthreads();
    if (tid == 0) {
        int m = sh_i[0];
        for (int w = 1; w < NA_THREADS / 32; ++w) m = min(m, sh_i[w]);
        sh_emin = m;
    }
    __syncthreads();
    const int32_t emin = sh_emin;
    int L = 1;
    while (L < R) L <<= 1;
    for (int r = tid; r < L; r += NA_THREADS) {
        double acc = 0.0;
        unsigned long long t = 0ull;
        if (r < R) {
            acc = 1.0;
            uint32_t d = (uint32_t)(E[r] - emin);
            while (d) {
                const int b = __ffs(d) - 1;
                acc = __dmul_rn(acc, qp.v[b]);
                d &= d - 1u;
            }
            t = (unsigned long long)__dmul_rn(acc, 4294967296.0);
            s->t[r] = t;
        }
        s->w[r] = acc;
    }
    __syncthreads();
    // Pairwise tree over slots padded with zeros to L: s_i <- s_2i + s_2i+1.
    double *src = s->w, *dst = s->w2;
    for (int len = L; len > 1; len >>= 1) {
        for (int i = tid; i < len / 2; i += NA_THREADS) dst[i] = __dadd_rn(src[2 * i], src[2 * i + 1]);
        __syncthreads();
        double *tmp = src;
        src = dst;
        dst = tmp;
    }
    // Exclusive prefix of t: contiguous chunks per thread, then across threads.
    const int chunk = (R + NA_THREADS - 1) / NA_THREADS;
    const int r0 = tid * chunk, r1 = min(R, r0 + chunk);
    unsigned long long loc = 0ull;
    for (int r = r0; r < r1; ++r) loc += s->t[r];
    unsigned long long inc = loc;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) sh_u[warp] = inc;
    __syncthreads();
    unsigned long long pre = inc - loc;
    for (int w = 0; w < warp; ++w) pre += sh_u[w];
    unsigned long long T = 0ull;
    for (int w = 0; w < NA_THREADS / 32; ++w) T += sh_u[w];
    const uint32_t o = pa::philox10(make_uint4(0u, 0u, k, pa::TAG_RESAMPLE), key0, key1).x;
    for (int r = r0; r < r1; ++r) {
        const unsigned long long P = pre;
        pre += s->t[r];
        const int32_t lo = na_count(P, R, T, o);
        const int32_t hi = na_count(P + s->t[r], R, T, o);
        for (int q = lo; q < hi; ++q) parent[q] = r;
        if (counts) counts[r] = hi - lo;
    }
    if (tid == 0) {
        s->A = src[0];
        s->T = T;
        s->emin = emin;
        s->o = o;
    }
}

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[64] = {};

}  // namespace

extern "C" int pa_resample_noalloc(const int32_t *energies, int32_t R, double beta_prev, double beta_k,
                                   uint64_t seed, int32_t k, int32_t *parent, int32_t *counts,
                                   pa_resample_result *out, void *stream) {
    if (!energies || !parent || R < 1 || R > NA_MAX_R || k < 0) return PA_EINVAL;
    if (!std::isfinite(beta_prev) || !std::isfinite(beta_k) || beta_prev < 0.0 || beta_k < beta_prev)
        return PA_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PA_ECUDA;
    void *base = nullptr;
    {
        // Set-up once per device, with that device current: host code only has a
        // stand-in for the __device__ array, so its device address is looked up.
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return PA_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        base = g_noalloc_ptr[dev];
    }
    NoallocScratch *s = reinterpret_cast<NoallocScratch *>(base);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    QPow qp;
    double sq = std::exp(-(beta_k - beta_prev));
    for (int b = 0; b < 32; ++b) {
        qp.v[b] = sq;
        sq = sq * sq;
    }
    k_resample_noalloc<<<1, NA_THREADS, 0, st>>>(energies, R, s, qp, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                 (uint32_t)k, parent, counts);
    if (cudaGetLastError() != cudaSuccess) return PA_ECUDA;
    if (out) {
        pa_resample_result res;
        if (cudaMemcpyAsync(&res.A, &s->A, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&res.T, &s->T, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&res.emin, &s->emin, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&res.o, &s->o, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return PA_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return PA_ECUDA;
        *out = res;
    }
    return PA_OK;
}
