// pa_internal.cuh -- internal declarations of libpa.so (not part of the ABI).
//
// Device layout of one anneal (vertices renumbered by colour; "position" p
// is a vertex's index in that order, np = n rounded up to 16):
//   spins  int8  [Rpad][np]   +1/-1, ping-pong pair (cur / next)
//   fields int16 [Rpad][np]   h_p = sum_j w_pj x_j, ping-pong pair
//   E      int32 [Rpad]       Ising energy of each replica, ping-pong pair
//   parent int32 [Rpad]       new slot -> old slot of the current step
// Rpad rounds R up to the replica block of the sweep kernel; padding slots
// copy themselves and are excluded from every reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pa {

// Full 32x32 -> 64-bit product (both halves from one wide multiply).
__host__ __device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi) {
#ifdef __CUDA_ARCH__
    unsigned long long p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
#else
    const uint64_t p = (uint64_t)a * b;
#endif
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

// Word w (0..3) of a Philox output.
__host__ __device__ __forceinline__ uint32_t word_of(const uint4 &v, uint32_t w) {
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplies by 0xD2511F53 / 0xCD9E8D57, high halves xored with the other
// counter words and the key; key advanced by 0x9E3779B9 / 0xBB67AE85.
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0, hi0, lo1, hi1;
        mul_wide(0xD2511F53u, c.x, lo0, hi0);
        mul_wide(0xCD9E8D57u, c.z, lo1, hi1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Stream tags in the top four bits of counter word 3.
constexpr uint32_t TAG_SWEEP = 0u << 28;
constexpr uint32_t TAG_RESAMPLE = 1u << 28;
constexpr uint32_t TAG_NONLOCAL = 2u << 28;
constexpr uint32_t TAG_INIT = 3u << 28;
constexpr uint32_t TAG_TAIL = 4u << 28;

// Metropolis uniform of an attempt (vertex vid, replica slot, step k, sweep
// s): its top 8 bits are byte (slot & 3) of word ((slot >> 2) & 3) of
// Philox(vid, slot >> 4, k, s), so one call serves 16 replicas; its low 24
// bits are the top 24 bits of word (slot & 3) of Philox(vid, slot >> 2, k,
// tag 4 | s). A move with threshold T (accept iff u < T) needs the low bits
// only when the top byte of u equals that of T (probability 1/256), so they
// are drawn on that path alone.
static __device__ __forceinline__ uint32_t sweep_tail_bits(uint32_t vid, uint32_t slot, uint32_t k, uint32_t s,
                                                uint32_t key0, uint32_t key1) {
    const uint4 v = philox10(make_uint4(vid, slot >> 2, k, TAG_TAIL | s), key0, key1);
    return word_of(v, slot & 3u) >> 8;
}

// Decision of an attempt with m >= 1 and threshold T given the top byte of
// its uniform (c3 = TAG_SWEEP | s): u < T.
static __device__ __forceinline__ bool accept_by_top_byte(uint32_t top, uint32_t T, uint32_t vid, uint32_t slot,
                                                   uint32_t k, uint32_t c3, uint32_t key0, uint32_t key1) {
    const uint32_t t8 = T >> 24;
    if (top != t8) return top < t8;
    return sweep_tail_bits(vid, slot, k, c3 & 0x0FFFFFFFu, key0, key1) < (T & 0xFFFFFFu);
}

constexpr int32_t EMIN_SENTINEL = 0x7F7F7F7F;  // byte-fillable "+infinity"
constexpr int RS_CHUNK = 256;                   // slots per resampling CTA (power of two)

struct GraphDev {
    int32_t n, np, ncol, mmax;
    const uint32_t *rp;   // [n+1] row pointers, position order
    const uint16_t *col;  // [2M] neighbour positions
    const int8_t *wt;     // [2M] weights or nullptr (all +1)
    const uint32_t *vid;  // [n] original vertex of each position
    const int32_t *cls;   // [ncol+1] colour class boundaries in positions
    const uint32_t *parity;  // [(np+31)/32] bit p = deg(p) & 1
    // Rows padded to multiples of 4 entries for 8-byte loads (packed kernel):
    // entry = neighbour position | 0x8000 if the weight is -1; padding entries
    // point at one of 32 scratch words after the np real ones.
    const uint32_t *prp;     // [n+1] row starts in units of 4 entries
    const uint2 *pcol;       // [prp[n]] four 16-bit entries each
    int32_t packed_ok;       // the padded encoding exists (np + 32 <= 32768)
    // Rows for the multi-spin-coded kernels (np <= 16384, degree <= 127), padded
    // to multiples of 4 entries: entry = 4 * neighbour position (the byte
    // offset of its word) | 1 if the weight is -1; padding entries point at the
    // row's own position (its word XOR itself counts nothing). mrp[p] = (row
    // start in units of 4 entries) << 8 | degree. nullptr when absent.
    const uint32_t *mrp;     // [n+1]
    const uint2 *mcol;       // [mrp[n] >> 8]
};

struct SweepArgs {
    GraphDev g;
    const int8_t *spins_in;
    const int16_t *fields_in;
    const int32_t *E_in;
    int8_t *spins_out;
    int16_t *fields_out;
    int32_t *E_out;
    const int32_t *parent;       // [Rpad]
    const uint32_t *tables;      // [ntables][mmax+1] acceptance thresholds
    const int32_t *tidx;         // [K] table used by step k
    const int32_t *active;       // [K] 0 = skip the step (adaptive end), may be null
    int32_t R, nblk, S, k;       // nblk: replica blocks of this launch
    int32_t blk_base;            // first replica block of this launch (multi-spin-coded kernels)
    uint32_t key0, key1;
    uint32_t rk0[10], rk1[10];   // Philox round keys key + r * (0x9E3779B9, 0xBB67AE85)
    int4 *best_rec;              // [all blocks] (E, step, sweep, slot) per replica block
    int8_t *best_cfg;            // [nblk][np] configuration of that record
    unsigned long long *accepts; // [K] accepted flips per step
    int32_t *sweep_emin;         // [K][S] minimum energy per sweep end
};

struct ResampleArgs {
    const int32_t *E;            // [Rpad] energies entering the step
    int32_t R, nch, k;
    uint32_t key0, key1;
    const double *qpow;          // [K][32] squarings of q_k, or per-dn table (adaptive)
    const int32_t *qsel;         // adaptive: row of qpow for step k (nullptr: row k)
    const int32_t *active;       // [K] or nullptr
    int32_t *emin;               // [K]
    double *partA;               // [nch]
    unsigned long long *partT;   // [nch]
    unsigned long long *tval;    // [Rpad]
    unsigned long long *ploc;    // [Rpad]
    int32_t *parent;             // [Rpad]
    double *recA;                // [K]
    unsigned long long *recT;    // [K]
    uint32_t *reco;              // [K]
    int32_t *counts;             // [K][R] or nullptr
    unsigned long long *stamp;   // [K+1] globaltimer at the start of each step
};

// Launchers (return cudaGetLastError()).
cudaError_t launch_init(const GraphDev &g, int8_t *spins, int32_t Rpad, uint32_t key0,
                        uint32_t key1, cudaStream_t st);
cudaError_t launch_fields(const GraphDev &g, const int8_t *spins, int16_t *fields, int32_t *E,
                          int32_t Rpad, cudaStream_t st);
// Minimum of the energies (and the step's start stamp), then weights + parents.
cudaError_t launch_rs_min(const ResampleArgs &a, cudaStream_t st);
cudaError_t launch_rs_rest(const ResampleArgs &a, cudaStream_t st);
cudaError_t launch_stamp(unsigned long long *stamp, cudaStream_t st);

struct SweepConfig {
    int G;          // replica groups of 4 per CTA (1 or 2)
    int field_bits; // 16, 8, 7 (packed spin + field byte), or 1 (multi-spin coded)
    int threads;
    int grid;
    size_t smem;
};
// Dynamic shared memory of one sweep CTA (G: 4-replica groups of the int8/int16 layouts;
// field_bits 1/2 multi-spin coded, 7 packed, 8/16 int8/int16 fields).
size_t sweep_smem_bytes(const GraphDev &g, int G, int field_bits, int threads);
cudaError_t sweep_configure(const GraphDev &g, int R, int G, int field_bits, int threads,
                            bool weighted, SweepConfig *cfg);
cudaError_t launch_sweep(const SweepConfig &cfg, const SweepArgs &a, cudaStream_t st);

}  // namespace pa
