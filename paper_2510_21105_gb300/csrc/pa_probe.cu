// pa_probe.cu -- pa_probe_peaks(): throughput probes that give the roofline
// denominators of the sweep kernels on the device they run on. The sweep is
// bound by integer issue (no tensor-core contraction, little DRAM traffic), so
// the probes measure, with register-only or shared-memory-only loops:
//   int_ops      32-bit integer instructions per second for a 1:1 mix of
//                multiply-adds (IMAD, FMA pipe) and three-input logic ops
//                (LOP3, ALU pipe), eight independent chains per thread;
//   philox       Philox4x32-10 output words per second (ten rounds per call,
//                no sharing between calls);
//   smem         shared-memory load bandwidth with conflict-free 16-byte loads.
// Each probe runs four 256-thread CTAs per SM and is timed with CUDA events;
// the best of three launches is kept.
#include <cuda_runtime.h>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 4;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_int(uint32_t seed, uint32_t mulc, uint32_t k, int iters,
                                                             uint32_t *sink) {
    uint32_t x[8], y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        x[j] = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (uint32_t)j;
        y[j] = blockIdx.x + 77u * (uint32_t)j;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            x[j] = x[j] * mulc + y[j];   // IMAD
            y[j] = y[j] ^ x[j] ^ k;      // LOP3
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc ^= x[j] + y[j];
    if (sink && acc == 0x12345678u) sink[0] = acc;   // keeps the chains live
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_philox(uint32_t key0, uint32_t key1, int iters,
                                                                uint32_t *sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < iters; i += 2) {
        const uint4 a = pa::philox10(make_uint4(t, (uint32_t)i, 7u, 0u), key0, key1);
        const uint4 b = pa::philox10(make_uint4(t, (uint32_t)i + 1u, 7u, 0u), key0, key1);
        acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
    }
    if (sink && acc == 0x12345678u) sink[0] = acc;
}

constexpr int SMEM_WORDS = 4096;   // 16 KB

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_smem(int iters, uint32_t *sink) {
    __shared__ __align__(16) uint32_t buf[SMEM_WORDS];
    for (int i = threadIdx.x; i < SMEM_WORDS; i += blockDim.x) buf[i] = (uint32_t)i * 2654435761u;
    __syncthreads();
    // Lanes read consecutive 16-byte words (no bank conflicts). The loads are
    // volatile so that the compiler keeps every one of them: the addresses
    // repeat every four iterations and nothing writes the buffer in the loop.
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    uint32_t acc = 0;
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        uint32_t w0, w1, w2, w3;
        asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3)
                     : "r"(base + 16u * (uint32_t)idx));
        acc ^= w0 ^ w1 ^ w2 ^ w3;
        idx = (idx + PROBE_THREADS) & (SMEM_WORDS / 4 - 1);
    }
    if (sink && acc == 0x12345678u) sink[0] = acc;
}

template <class F>
double best_ms(F launch, cudaStream_t st, int *err) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        *err = 1;
        return 0.0;
    }
    launch();   // warm-up
    double best = 1e30;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) *err = 1;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f && ms < best) best = ms;
    }
    if (cudaGetLastError() != cudaSuccess) *err = 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

extern "C" int pa_probe_peaks(pa_peaks *out, void *stream) {
    if (!out) return PA_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return PA_ECUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The probes store their checksum only through a non-null sink, so passing
    // NULL keeps every chain live (the compiler cannot see the pointer) while
    // nothing is ever written.
    uint32_t *sink = nullptr;
    const int grid = sms * PROBE_CTAS_PER_SM;
    const double threads = (double)grid * PROBE_THREADS;
    int err = 0;
    const int it_int = 1 << 14, it_ph = 1 << 11, it_sm = 1 << 15;
    const double ms_int = best_ms([&] { k_probe_int<<<grid, PROBE_THREADS, 0, st>>>(12345u, 0x2545F491u, 0x5bd1e995u,
                                                                                  it_int, sink); }, st, &err);
    const double ms_ph = best_ms([&] { k_probe_philox<<<grid, PROBE_THREADS, 0, st>>>(0xA511E9B3u, 0x3C6EF372u,
                                                                                    it_ph, sink); }, st, &err);
    const double ms_sm = best_ms([&] { k_probe_smem<<<grid, PROBE_THREADS, 0, st>>>(it_sm, sink); }, st, &err);
    if (err || ms_int <= 0.0 || ms_ph <= 0.0 || ms_sm <= 0.0) return PA_ECUDA;
    out->int_ops_per_s = threads * it_int * 16.0 / (ms_int * 1e-3);
    out->philox_words_per_s = threads * it_ph * 4.0 / (ms_ph * 1e-3);
    out->smem_bytes_per_s = threads * it_sm * 16.0 / (ms_sm * 1e-3);
    out->sms = sms;
    return PA_OK;
}
