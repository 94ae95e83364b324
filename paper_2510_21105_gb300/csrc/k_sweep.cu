// k_sweep.cu -- colour-ordered Metropolis sweeps of PAMC (Sec. 3 of arXiv
// 2510.21105; the paper names the method but not the sweep, so the rule is
// the library's reading: standard Metropolis on the Ising form of Eq. 1).
//
// One CTA holds a block of B = 4G replicas in shared memory while it runs all
// S sweeps of one temperature step on them:
//   S_sm[p][g]  uint32: int8 spins of replicas 4g..4g+3 at position p
//   H_sm[p][g]  local fields of the same replicas, biased to unsigned:
//               16-bit: two uint32 words (replicas 0,1 | 2,3), h + 32768
//                8-bit: one uint32 word, h + 128 (max degree <= 127)
// A colour class is an independent set, so all of its positions update in
// parallel (one thread per (position, group)); the accepted flips push
// +-2 into the neighbours' fields with one packed 32-bit shared atomic per
// neighbour and group (the bias keeps every lane non-negative, so the packed
// add never carries across lanes). The top bytes of the group's four
// uniforms are the bytes of one word of Philox(counter = (vertex, slot/16,
// step, sweep)): byte q of word (slot/4) % 4 belongs to slot 4*(slot/4) + q;
// the low 24 bits are drawn only when a top byte ties with the threshold's.
// The block is loaded from the parents chosen by the resampling (the copy of
// the resampling is fused into this load) and written to the next buffers.
#include <cooperative_groups.h>

#include <mutex>
#include <unordered_map>

#include "pa_internal.cuh"

namespace pa {
namespace {

__device__ __forceinline__ void transpose4x4_bytes(uint32_t w0, uint32_t w1, uint32_t w2,
                                                   uint32_t w3, uint32_t o[4]) {
    const uint32_t a_lo = __byte_perm(w0, w1, 0x5140);
    const uint32_t a_hi = __byte_perm(w0, w1, 0x7362);
    const uint32_t b_lo = __byte_perm(w2, w3, 0x5140);
    const uint32_t b_hi = __byte_perm(w2, w3, 0x7362);
    o[0] = __byte_perm(a_lo, b_lo, 0x5410);
    o[1] = __byte_perm(a_lo, b_lo, 0x7632);
    o[2] = __byte_perm(a_hi, b_hi, 0x5410);
    o[3] = __byte_perm(a_hi, b_hi, 0x7632);
}

// Byte permute with sign replication: each selector nibble with bit 3 set
// fills its result byte with the top bit of the selected byte.
__device__ __forceinline__ uint32_t prmt_sign(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Entry i of a decision table in 16-bit lanes (the multi-spin-coded and the
// packed kernels): E(m) in both halves, m = i - 32 for counts of |m| <= 31
// kept as byte offsets 4m + 128, else m = i - 128 (word index). With the top
// byte of the uniform, lane = 128 top + E is below 0x8000 iff the move is
// accepted, 0x8000 exactly on a tie that the low bits decide.
__device__ __forceinline__ uint32_t msc_entry(int i, bool pk, const uint32_t *tab, int mmax) {
    const int m = pk ? i - 32 : i - 128;
    uint32_t e = 1u;   // m <= 0: always accepted
    if (m > 0) {
        const uint32_t T = m <= mmax ? tab[m] : 0u;
        e = T == 0u ? 0x8040u : 0x8000u - 128u * (T >> 24) + ((T & 0xFFFFFFu) == 0u ? 64u : 0u);
    }
    return e * 0x00010001u;
}

template <int G, int FB, bool WEIGHTED>
__device__ __forceinline__ void sweep_item(uint32_t *__restrict__ Ssm, uint32_t *__restrict__ Hsm,
                                           const uint32_t *__restrict__ Tt, const SweepArgs &a,
                                           int p, int g, uint32_t c1, uint32_t c3, uint32_t vmask,
                                           int dE[4], uint32_t &nacc) {
    const int widx = p * G + g;
    const uint32_t sw = Ssm[widx];
    uint32_t hw0, hw1 = 0;
    if (FB == 16) {
        const uint2 hv = reinterpret_cast<const uint2 *>(Hsm)[widx];
        hw0 = hv.x;
        hw1 = hv.y;
    } else {
        hw0 = Hsm[widx];
    }
    int m[4], x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        x[q] = (int)(int8_t)(sw >> (8 * q));
        int h;
        if (FB == 16)
            h = (int)(((q < 2 ? hw0 : hw1) >> (16 * (q & 1))) & 0xFFFFu) - 32768;
        else
            h = (int)((hw0 >> (8 * q)) & 0xFFu) - 128;
        m[q] = x[q] > 0 ? -h : h;   // dE = -2 x h = 2m
    }
    // Top bytes of the four uniforms: word c1 & 3 of the call of slots 16 (c1 >> 2) ..
    const uint32_t vid = __ldg(&a.g.vid[p]);
    const uint32_t uw = word_of(philox10(make_uint4(vid, c1 >> 2, (uint32_t)a.k, c3), a.key0, a.key1), c1 & 3u);
    uint32_t acc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool ok = (m[q] <= 0) || accept_by_top_byte((uw >> (8 * q)) & 0xFFu, Tt[min(m[q], a.g.mmax)], vid,
                                                          4u * c1 + q, (uint32_t)a.k, c3, a.key0, a.key1);
        acc |= (uint32_t)ok << q;
    }
    if (acc) {
        uint32_t flip = 0;
        int d[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool f = (acc >> q) & 1u;
            flip |= f ? (0xFEu << (8 * q)) : 0u;
            dE[q] += f ? 2 * m[q] : 0;
            d[q] = f ? -2 * x[q] : 0;
        }
        Ssm[widx] = sw ^ flip;
        nacc += __popc(acc & vmask);
        uint32_t D0, D1 = 0;
        if (FB == 16) {
            D0 = (uint32_t)(d[0] + d[1] * 65536);
            D1 = (uint32_t)(d[2] + d[3] * 65536);
        } else {
            D0 = (uint32_t)(d[0] + d[1] * 256 + d[2] * 65536 + d[3] * 16777216);
        }
        const uint32_t e0 = __ldg(&a.g.rp[p]), e1 = __ldg(&a.g.rp[p + 1]);
        for (uint32_t e = e0; e < e1; ++e) {
            const int j = __ldg(&a.g.col[e]);
            uint32_t s0 = D0, s1 = D1;
            if (WEIGHTED) {
                if (__ldg(&a.g.wt[e]) < 0) {
                    s0 = 0u - D0;
                    s1 = 0u - D1;
                }
            }
            if (FB == 16) {
                atomicAdd(&Hsm[2 * (j * G + g)], s0);
                atomicAdd(&Hsm[2 * (j * G + g) + 1], s1);
            } else {
                atomicAdd(&Hsm[j * G + g], s0);
            }
        }
    }
}

template <int G, int FB, bool WEIGHTED>
__global__ void __launch_bounds__(1024) k_sweep(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    // A step after the adaptive schedule has ended only carries the population over.
    const bool act = !a.active || a.active[a.k];
    const int nsweeps = act ? a.S : 0;
    const int np = a.g.np;
    constexpr int HW = (FB == 16) ? 2 : 1;
    uint32_t *Ssm = reinterpret_cast<uint32_t *>(smem);
    uint32_t *Hsm = Ssm + (size_t)np * G;
    uint32_t *Tt = Hsm + (size_t)np * G * HW;
    const int tsz = (a.g.mmax + 1 + 3) & ~3;
    int32_t *cls = reinterpret_cast<int32_t *>(Tt + tsz);
    const int csz = (a.g.ncol + 1 + 3) & ~3;
    int32_t *Eacc = cls + csz;          // [4G]
    int32_t *PS = Eacc + 4 * G;         // [4G] parent slot of each replica
    int32_t *misc = PS + 4 * G;         // best E, step, sweep, slot, copy-from (q+1), changed

    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    const uint32_t *tab = a.tables + (size_t)a.tidx[a.k] * (a.g.mmax + 1);
    for (int i = tid; i <= a.g.mmax; i += NT) Tt[i] = tab[i];
    for (int i = tid; i <= a.g.ncol; i += NT) cls[i] = a.g.cls[i];
    const int gthr = tid % G;   // NT is a multiple of 32, so each thread keeps one group

    for (int blk = blockIdx.x; blk < a.nblk; blk += gridDim.x) {
        const int slot0 = blk * 4 * G;
        if (tid < 4 * G) PS[tid] = act ? a.parent[slot0 + tid] : slot0 + tid;
        if (tid == 0) {
            const int4 br = a.best_rec[blk];
            misc[0] = br.x; misc[1] = br.y; misc[2] = br.z; misc[3] = br.w;
            misc[4] = 0; misc[5] = 0;
        }
        __syncthreads();
        if (tid < 4 * G) Eacc[tid] = a.E_in[PS[tid]];
        // Load the block, transposing replica rows into position-major words.
        for (int idx = tid; idx < (np >> 2) * G; idx += NT) {
            const int g = idx % G, c = idx / G;
            uint32_t w[4];
            uint2 f[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const size_t row = (size_t)PS[4 * g + q] * np + 4 * c;
                w[q] = __ldg(reinterpret_cast<const uint32_t *>(a.spins_in + row));
                f[q] = __ldg(reinterpret_cast<const uint2 *>(a.fields_in + row));
            }
            uint32_t o[4];
            transpose4x4_bytes(w[0], w[1], w[2], w[3], o);
#pragma unroll
            for (int j = 0; j < 4; ++j) Ssm[(4 * c + j) * G + g] = o[j];
            if (FB == 16) {
                uint2 *H2 = reinterpret_cast<uint2 *>(Hsm);
                H2[(4 * c + 0) * G + g] = make_uint2(__byte_perm(f[0].x, f[1].x, 0x5410) ^ 0x80008000u,
                                                     __byte_perm(f[2].x, f[3].x, 0x5410) ^ 0x80008000u);
                H2[(4 * c + 1) * G + g] = make_uint2(__byte_perm(f[0].x, f[1].x, 0x7632) ^ 0x80008000u,
                                                     __byte_perm(f[2].x, f[3].x, 0x7632) ^ 0x80008000u);
                H2[(4 * c + 2) * G + g] = make_uint2(__byte_perm(f[0].y, f[1].y, 0x5410) ^ 0x80008000u,
                                                     __byte_perm(f[2].y, f[3].y, 0x5410) ^ 0x80008000u);
                H2[(4 * c + 3) * G + g] = make_uint2(__byte_perm(f[0].y, f[1].y, 0x7632) ^ 0x80008000u,
                                                     __byte_perm(f[2].y, f[3].y, 0x7632) ^ 0x80008000u);
            } else {
                const uint32_t px01 = __byte_perm(f[0].x, f[1].x, 0x6420);
                const uint32_t px23 = __byte_perm(f[2].x, f[3].x, 0x6420);
                const uint32_t py01 = __byte_perm(f[0].y, f[1].y, 0x6420);
                const uint32_t py23 = __byte_perm(f[2].y, f[3].y, 0x6420);
                Hsm[(4 * c + 0) * G + g] = __byte_perm(px01, px23, 0x6420) ^ 0x80808080u;
                Hsm[(4 * c + 1) * G + g] = __byte_perm(px01, px23, 0x7531) ^ 0x80808080u;
                Hsm[(4 * c + 2) * G + g] = __byte_perm(py01, py23, 0x6420) ^ 0x80808080u;
                Hsm[(4 * c + 3) * G + g] = __byte_perm(py01, py23, 0x7531) ^ 0x80808080u;
            }
        }
        __syncthreads();

        uint32_t vmask = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) vmask |= (slot0 + 4 * gthr + q < a.R) ? (1u << q) : 0u;
        const uint32_t c1 = (uint32_t)(blk * G + gthr);
        uint32_t nacc = 0;
        for (int s = 0; s < nsweeps; ++s) {
            const uint32_t c3 = TAG_SWEEP | (uint32_t)s;
            int dE[4] = {0, 0, 0, 0};
            for (int c = 0; c < a.g.ncol; ++c) {
                const int p0 = cls[c];
                const int cnt = (cls[c + 1] - p0) * G;
                for (int idx = tid; idx < cnt; idx += NT)
                    sweep_item<G, FB, WEIGHTED>(Ssm, Hsm, Tt, a, p0 + idx / G, gthr, c1, c3, vmask,
                                                dE, nacc);
                __syncthreads();
            }
            // Energies after sweep s: reduce the per-thread changes of each replica.
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int v = dE[q];
#pragma unroll
                for (int off = G; off < 32; off <<= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
                if (lane < G && v != 0) atomicAdd(&Eacc[4 * lane + q], v);
            }
            __syncthreads();
            if (tid == 0) {
                int bq = -1, bE = 0x7FFFFFFF;
                for (int q = 0; q < 4 * G; ++q)
                    if (slot0 + q < a.R && Eacc[q] < bE) { bE = Eacc[q]; bq = q; }
                misc[4] = 0;
                if (bq >= 0) {
                    atomicMin(&a.sweep_emin[(size_t)a.k * a.S + s], bE);
                    if (bE < misc[0]) {
                        misc[0] = bE; misc[1] = a.k; misc[2] = s; misc[3] = slot0 + bq;
                        misc[4] = bq + 1; misc[5] = 1;
                    }
                }
            }
            __syncthreads();
            if (misc[4]) {   // block-uniform: copy the new best configuration
                const int q = misc[4] - 1, g = q >> 2, sh = 8 * (q & 3);
                uint32_t *dst = reinterpret_cast<uint32_t *>(a.best_cfg + (size_t)blk * np);
                for (int c = tid; c < (np >> 2); c += NT) {
                    uint32_t v = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) v |= ((Ssm[(4 * c + j) * G + g] >> sh) & 0xFFu) << (8 * j);
                    dst[c] = v;
                }
                __syncthreads();
            }
        }
        // Store the block to the next population buffers.
        for (int idx = tid; idx < (np >> 2) * G; idx += NT) {
            const int g = idx % G, c = idx / G;
            uint32_t o[4];
            transpose4x4_bytes(Ssm[(4 * c + 0) * G + g], Ssm[(4 * c + 1) * G + g],
                               Ssm[(4 * c + 2) * G + g], Ssm[(4 * c + 3) * G + g], o);
            uint2 f[4];
            if (FB == 16) {
                const uint2 *H2 = reinterpret_cast<const uint2 *>(Hsm);
                const uint2 h0 = H2[(4 * c + 0) * G + g], h1 = H2[(4 * c + 1) * G + g];
                const uint2 h2 = H2[(4 * c + 2) * G + g], h3 = H2[(4 * c + 3) * G + g];
                const uint32_t L0 = h0.x ^ 0x80008000u, L1 = h1.x ^ 0x80008000u;
                const uint32_t L2 = h2.x ^ 0x80008000u, L3 = h3.x ^ 0x80008000u;
                const uint32_t U0 = h0.y ^ 0x80008000u, U1 = h1.y ^ 0x80008000u;
                const uint32_t U2 = h2.y ^ 0x80008000u, U3 = h3.y ^ 0x80008000u;
                f[0] = make_uint2(__byte_perm(L0, L1, 0x5410), __byte_perm(L2, L3, 0x5410));
                f[1] = make_uint2(__byte_perm(L0, L1, 0x7632), __byte_perm(L2, L3, 0x7632));
                f[2] = make_uint2(__byte_perm(U0, U1, 0x5410), __byte_perm(U2, U3, 0x5410));
                f[3] = make_uint2(__byte_perm(U0, U1, 0x7632), __byte_perm(U2, U3, 0x7632));
            } else {
                uint32_t P[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) P[j] = Hsm[(4 * c + j) * G + g] ^ 0x80808080u;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int h[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) h[j] = (int)(int8_t)(P[j] >> (8 * q));
                    f[q] = make_uint2(((uint32_t)h[0] & 0xFFFFu) | ((uint32_t)h[1] << 16),
                                      ((uint32_t)h[2] & 0xFFFFu) | ((uint32_t)h[3] << 16));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const size_t row = (size_t)(slot0 + 4 * g + q) * np + 4 * c;
                *reinterpret_cast<uint32_t *>(a.spins_out + row) = o[q];
                *reinterpret_cast<uint2 *>(a.fields_out + row) = f[q];
            }
        }
        if (tid < 4 * G) a.E_out[slot0 + tid] = Eacc[tid];
        if (tid == 0 && misc[5]) a.best_rec[blk] = make_int4(misc[0], misc[1], misc[2], misc[3]);
        const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, nacc);
        if (act && lane == 0 && wsum) atomicAdd(&a.accepts[a.k], (unsigned long long)wsum);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Packed variant: one byte per (position, replica) holds the spin in bit 0 and
// the biased local field in bits 1..7. Because h_p = sum of deg(p) terms +-1,
// h_p + 128 has the parity of deg(p), so its low bit is redundant and is
// replaced by the spin bit:  byte = ((h + 128) & ~1) | s,  s = (x == +1).
// Needs max degree <= 127. Flipping a spin toggles bit 0; a neighbour flip
// adds +-2 to the byte (bit 0 untouched), four replicas per packed atomic.
// With m = -x h and mb = m + 128 per byte:
//   hb = (b & 0xFE..) | par,  M = s * 0xFF,  mb = (hb ^ M) + s
// (for s = 1 this is the bytewise negation 256 - hb; hb >= 1 so no carry).
// A move is accepted iff mb <= 128 (m <= 0) or u < T[m].
struct PkItem {
    uint32_t b, mb, smask, acc;
};

// Ties of the top byte in a packed item (rare): the low 24 bits of the
// uniform decide.
__device__ __forceinline__ uint32_t pk_settle_ties(const SweepArgs &a, uint32_t acc, uint32_t tie, uint32_t mb,
                                                uint32_t vid, uint32_t c1, uint32_t c3) {
    const uint32_t *tab = a.tables + (size_t)a.tidx[a.k] * (a.g.mmax + 1);
    do {
        const int q = __ffs(tie) - 1;
        tie &= tie - 1u;
        const uint32_t T = __ldg(&tab[(int)((mb >> (8 * q)) & 0xFFu) - 128]);
        if (sweep_tail_bits(vid, 4u * c1 + q, (uint32_t)a.k, c3, a.key0, a.key1) < (T & 0xFFFFFFu)) acc |= 1u << q;
    } while (tie);
    return acc;
}

__device__ __forceinline__ void pk_decide(const uint32_t *__restrict__ Bsm, const uint32_t *__restrict__ T256,
                                          const uint32_t *__restrict__ Psm, const SweepArgs &a, int p,
                                          uint32_t c1, uint32_t c3, PkItem &it) {
    const uint32_t vid = __ldg(&a.g.vid[p]);
    const uint32_t b = Bsm[p];
    const uint32_t par = (Psm[p >> 5] >> (p & 31)) & 1u;
    const uint32_t smask = b & 0x01010101u;
    const uint32_t hb = (b & 0xFEFEFEFEu) | (par * 0x01010101u);
    const uint32_t mb = (hb ^ (smask * 0xFFu)) + smask;
    const uint32_t uw = word_of(philox10(make_uint4(vid, c1 >> 2, (uint32_t)a.k, c3), a.key0, a.key1), c1 & 3u);
    // The four decisions in 16-bit lanes, as in the multi-spin-coded item.
    const uint32_t e0 = T256[mb & 0xFFu], e1 = T256[(mb >> 8) & 0xFFu];
    const uint32_t e2 = T256[(mb >> 16) & 0xFFu], e3 = T256[mb >> 24];
    const uint32_t slo = __byte_perm(uw, 0u, 0x4140u) * 128u + __byte_perm(e0, e1, 0x5410u);
    const uint32_t shi = __byte_perm(uw, 0u, 0x4342u) * 128u + __byte_perm(e2, e3, 0x5410u);
    const uint32_t RT = prmt_sign(slo, shi, 0xFDB9u);                               // reject or tie
    const uint32_t RS = prmt_sign(slo - 0x00010001u, shi - 0x00010001u, 0xFDB9u);   // reject
    uint32_t acc = (((~RT >> 7) & 0x01010101u) * 0x01020408u) >> 24;       // bit q: replica q accepted
    uint32_t tie = ((((RT & ~RS) >> 7) & 0x01010101u) * 0x01020408u) >> 24;
    if (tie) acc = pk_settle_ties(a, acc, tie, mb, vid, c1, c3);   // rare
    it.b = b;
    it.mb = mb;
    it.smask = smask;
    it.acc = acc;
}

// Own word, energy and acceptance bookkeeping of an item; returns the packed
// field change D of its neighbours (0 if nothing was accepted).
__device__ __forceinline__ uint32_t pk_commit_self(uint32_t *__restrict__ Bsm, int p, const PkItem &it,
                                                   uint32_t vmask, int dE[4], uint32_t &nacc) {
    if (!it.acc) return 0u;
    const uint32_t a01 = (it.acc * 0x00204081u) & 0x01010101u;   // bit q -> bit 8q
    Bsm[p] = it.b ^ a01;
    nacc += __popc(it.acc & vmask);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        dE[q] += ((it.acc >> q) & 1u) ? 2 * ((int)((it.mb >> (8 * q)) & 0xFFu) - 128) : 0;
    // field change of the neighbours: -2 x_q per accepted replica q
    return ((a01 & ~it.smask) << 1) - ((a01 & it.smask) << 1);
}

// Per-warp ring of accepted items (position, D) awaiting their neighbour
// updates; a full round gives every lane one item, so the row walks run with
// all lanes busy instead of with the few lanes that happened to accept.
constexpr int PK_QCAP = 64;   // backlog < 32 + 32 after each drain

__device__ __forceinline__ void pk_enqueue(uint2 *__restrict__ Q, uint32_t &qtail, int p, uint32_t D,
                                           int lane) {
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, D != 0u);
    if (D) {
        const uint32_t rank = __popc(bal & ((1u << lane) - 1u));
        Q[(qtail + rank) & (PK_QCAP - 1)] = make_uint2((uint32_t)p, D);
    }
    qtail += __popc(bal);
}

template <bool WEIGHTED>
__device__ __forceinline__ void pk_round(uint32_t *__restrict__ Bsm, const uint2 *__restrict__ Q,
                                         uint32_t qhead, uint32_t count, const SweepArgs &a, int lane) {
    __syncwarp();
    if ((uint32_t)lane < count) {
        const uint2 ent = Q[(qhead + lane) & (PK_QCAP - 1)];
        const uint32_t D = ent.y;
        const uint32_t e0 = __ldg(&a.g.prp[ent.x]), e1 = __ldg(&a.g.prp[ent.x + 1]);
        for (uint32_t e = e0; e < e1; ++e) {
            const uint2 v = __ldg(&a.g.pcol[e]);
            const uint32_t idx[4] = {v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (WEIGHTED)
                    atomicAdd(&Bsm[idx[t] & 0x7FFFu], (idx[t] & 0x8000u) ? 0u - D : D);
                else
                    atomicAdd(&Bsm[idx[t]], D);
            }
        }
    }
    __syncwarp();
}

template <bool WEIGHTED, int NTB, int MINB>
__global__ void __launch_bounds__(NTB, MINB) k_sweep_packed(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const bool act = !a.active || a.active[a.k];
    const int nsweeps = act ? a.S : 0;
    const int np = a.g.np;
    uint32_t *Bsm = reinterpret_cast<uint32_t *>(smem);          // [np + 32], last 32 are scratch
    uint32_t *T256 = Bsm + np + 32;                                 // [256] decision entries by m + 128
    int32_t *cls = reinterpret_cast<int32_t *>(T256 + 256);
    const int csz = (a.g.ncol + 1 + 3) & ~3;
    int32_t *Eacc = cls + csz;      // [4]
    int32_t *PS = Eacc + 4;         // [4]
    int32_t *misc = PS + 4;         // best E, step, sweep, slot, copy-from (q+1), changed
    uint32_t *Psm = reinterpret_cast<uint32_t *>(misc + 8);         // degree parity bits
    const int npw = (np + 31) >> 5;
    uint2 *Qall = reinterpret_cast<uint2 *>(Psm + ((npw + 1) & ~1));  // [NT/32][PK_QCAP]

    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    uint2 *Q = Qall + (size_t)(tid >> 5) * PK_QCAP;
    const uint32_t *tab = a.tables + (size_t)a.tidx[a.k] * (a.g.mmax + 1);
    for (int i = tid; i < 256; i += NT) T256[i] = msc_entry(i, false, tab, a.g.mmax);   // by m + 128
    for (int i = tid; i <= a.g.ncol; i += NT) cls[i] = a.g.cls[i];
    for (int i = tid; i < npw; i += NT) Psm[i] = a.g.parity[i];

    for (int blk = blockIdx.x; blk < a.nblk; blk += gridDim.x) {
        const int slot0 = blk * 4;
        if (tid < 4) PS[tid] = act ? a.parent[slot0 + tid] : slot0 + tid;
        if (tid == 0) {
            const int4 br = a.best_rec[blk];
            misc[0] = br.x; misc[1] = br.y; misc[2] = br.z; misc[3] = br.w;
            misc[4] = 0; misc[5] = 0;
        }
        __syncthreads();
        if (tid < 4) Eacc[tid] = a.E_in[PS[tid]];
        // Load: int8 spins + int16 fields of four replica rows -> packed bytes.
        for (int c = tid; c < (np >> 2); c += NT) {
            uint32_t w[4];
            uint2 f[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const size_t row = (size_t)PS[q] * np + 4 * c;
                w[q] = __ldg(reinterpret_cast<const uint32_t *>(a.spins_in + row));
                f[q] = __ldg(reinterpret_cast<const uint2 *>(a.fields_in + row));
            }
            uint32_t o[4];
            transpose4x4_bytes(w[0], w[1], w[2], w[3], o);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t word = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t hv = j < 2 ? f[q].x : f[q].y;
                    const uint32_t h128 = ((hv >> (16 * (j & 1))) + 128u) & 0xFFu;   // h + 128
                    const uint32_t sbit = ((o[j] >> (8 * q)) & 0xFFu) == 1u ? 1u : 0u;
                    word |= ((h128 & 0xFEu) | sbit) << (8 * q);
                }
                Bsm[4 * c + j] = word;
            }
        }
        __syncthreads();

        uint32_t vmask = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) vmask |= (slot0 + q < a.R) ? (1u << q) : 0u;
        const uint32_t c1 = (uint32_t)blk;
        uint32_t nacc = 0;
        for (int s = 0; s < nsweeps; ++s) {
            const uint32_t c3 = TAG_SWEEP | (uint32_t)s;
            int dE[4] = {0, 0, 0, 0};
            for (int c = 0; c < a.g.ncol; ++c) {
                const int p0 = cls[c], p1 = cls[c + 1];
                uint32_t qhead = 0, qtail = 0;   // warp-uniform
                for (int base = p0; base < p1; base += 2 * NT) {   // trip count uniform in the CTA
                    const int pA = base + tid, pB = pA + NT;
                    PkItem A, Bi;
                    A.acc = 0;
                    Bi.acc = 0;
                    if (pA < p1) pk_decide(Bsm, T256, Psm, a, pA, c1, c3, A);
                    if (pB < p1) pk_decide(Bsm, T256, Psm, a, pB, c1, c3, Bi);
                    const uint32_t DA = pk_commit_self(Bsm, pA, A, vmask, dE, nacc);
                    const uint32_t DB = pk_commit_self(Bsm, pB, Bi, vmask, dE, nacc);
                    pk_enqueue(Q, qtail, pA, DA, lane);
                    if (qtail - qhead >= 32u) {
                        pk_round<WEIGHTED>(Bsm, Q, qhead, 32u, a, lane);
                        qhead += 32u;
                    }
                    pk_enqueue(Q, qtail, pB, DB, lane);
                    if (qtail - qhead >= 32u) {
                        pk_round<WEIGHTED>(Bsm, Q, qhead, 32u, a, lane);
                        qhead += 32u;
                    }
                }
                if (qtail != qhead) pk_round<WEIGHTED>(Bsm, Q, qhead, qtail - qhead, a, lane);
                __syncthreads();
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int v = __reduce_add_sync(0xFFFFFFFFu, dE[q]);
                if (lane == 0 && v != 0) atomicAdd(&Eacc[q], v);
            }
            __syncthreads();
            if (tid == 0) {
                int bq = -1, bE = 0x7FFFFFFF;
                for (int q = 0; q < 4; ++q)
                    if (slot0 + q < a.R && Eacc[q] < bE) { bE = Eacc[q]; bq = q; }
                misc[4] = 0;
                if (bq >= 0) {
                    atomicMin(&a.sweep_emin[(size_t)a.k * a.S + s], bE);
                    if (bE < misc[0]) {
                        misc[0] = bE; misc[1] = a.k; misc[2] = s; misc[3] = slot0 + bq;
                        misc[4] = bq + 1; misc[5] = 1;
                    }
                }
            }
            __syncthreads();
            if (misc[4]) {
                const int sh = 8 * (misc[4] - 1);
                uint32_t *dst = reinterpret_cast<uint32_t *>(a.best_cfg + (size_t)blk * np);
                for (int c = tid; c < (np >> 2); c += NT) {
                    uint32_t v = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t sb = (Bsm[4 * c + j] >> sh) & 1u;
                        const bool real = 4 * c + j < a.g.n;
                        v |= (real ? (sb ? 0x01u : 0xFFu) : 0u) << (8 * j);
                    }
                    dst[c] = v;
                }
                __syncthreads();
            }
        }
        // Store: packed bytes -> int8 spins + int16 fields of the next buffers.
        for (int c = tid; c < (np >> 2); c += NT) {
            uint32_t sp[4] = {0u, 0u, 0u, 0u};
            uint32_t fx[4] = {0u, 0u, 0u, 0u}, fy[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = 4 * c + j;
                const uint32_t word = Bsm[p];
                const uint32_t pb = (Psm[p >> 5] >> (p & 31)) & 1u;
                const bool real = p < a.g.n;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t byte = (word >> (8 * q)) & 0xFFu;
                    const uint32_t sv = real ? ((byte & 1u) ? 0x01u : 0xFFu) : 0u;
                    const int h = real ? (int)((byte & 0xFEu) | pb) - 128 : 0;
                    sp[q] |= sv << (8 * j);
                    if (j < 2) fx[q] |= ((uint32_t)h & 0xFFFFu) << (16 * j);
                    else fy[q] |= ((uint32_t)h & 0xFFFFu) << (16 * (j - 2));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const size_t row = (size_t)(slot0 + q) * np + 4 * c;
                *reinterpret_cast<uint32_t *>(a.spins_out + row) = sp[q];
                *reinterpret_cast<uint2 *>(a.fields_out + row) = make_uint2(fx[q], fy[q]);
            }
        }
        if (tid < 4) a.E_out[slot0 + tid] = Eacc[tid];
        if (tid == 0 && misc[5]) a.best_rec[blk] = make_int4(misc[0], misc[1], misc[2], misc[3]);
        const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, nacc);
        if (act && lane == 0 && wsum) atomicAdd(&a.accepts[a.k], (unsigned long long)wsum);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Multi-spin-coded variant: W[p] holds the spins of 32 replicas (slots
// 32*blk .. 32*blk+31) at position p, 1 for +1. Replica 4g + q (group g of
// the Philox call that serves it, word q) sits at bit 8q + g, so that a
// group's four replicas are one bit of each byte. No fields are kept:
// an item (p, word) XORs its word with each neighbour's word (and with all
// ones for a -1 weight), so bit r of d_j is 1 iff the bond (p, j) contributes
// +1 to m_r = -x_p h_p; a bit-sliced counter over the neighbours (carry-save
// adders, four bonds per step) gives c_r and m_r = 2 c_r - deg(p). An 8 x 8
// bit transpose in every byte lane turns the counter planes into one byte per
// replica, group by group. The uniforms of the group's four replicas have
// their top bytes in one Philox word (word g & 3 of the call of slots
// 16 (slot >> 4) ..): byte q belongs to replica 4g + q, the same byte as its
// count. With |m| <= 31 the count byte holds 4m + 128, which is also the byte
// offset of the entry of m in a table kept at the start of shared memory, so
// the lookup needs no address arithmetic (wider counts: m + 128, a word index).
// An entry holds a 16-bit value E(m) in both halves. Two replicas are decided
// by one 32-bit multiply-add in 16-bit lanes, lane = 128 top + E(m):
//   E = 0x8000 - 128 t8 (t8 = T[m] >> 24):  lane < 0x8000 iff top < t8 (accept),
//                                           lane = 0x8000 iff top = t8 (tie),
//   + 64 when T[m] has no low bits (a tie rejects), 0x8040 when T[m] = 0,
//   1 for m <= 0 (always accepted).
// Every lane stays in [1, 0xFFC0], so lanes never carry into each other; bit
// 15 of a lane is "reject or tie" and bit 15 of lane - 1 is "reject". A byte
// permute replicating those sign bits turns the four lanes of a group into
// byte masks. A tie (probability 1/256 per uncertain attempt) is settled by
// the low 24 bits of the uniform, drawn only then: the ties of a warp's items
// are queued and settled by all 32 lanes together before the class barrier
// (one tail Philox call per lane instead of one per tying lane while the
// others wait). Accepted replicas flip with one XOR.
__device__ __forceinline__ int msc_bit(int r) {   // bit of replica r = 4g + q in a word
    return 8 * (r & 3) + (r >> 2);
}

// Rows <-> bit words for 4 positions 4c .. 4c+3. A spin byte is 0x01 (+1) or
// 0xFF (-1), 0 on padding. Load: per group g the four rows 4g + q give a word
// y whose byte j holds, in bit q, replica 4g + q at position 4c + j; the
// multiply by 0x00204081 spreads that nibble so that bit q lands on bit 8q
// (the four shifted copies do not overlap, so nothing carries), and the shift
// by g puts it on bit 8q + g of the position's word. Store: the inverse, with
// byte j of the row word = 0x01 or 0xFF from the spread bit d (0xFF ^ 0xFE d)
// and 0 on padding positions.
__device__ __forceinline__ void msc_pack_rows(const int8_t *spins_in, const int32_t *PS, int np, int c,
                                              uint32_t (&w4)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) w4[j] = 0u;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        uint32_t y = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t v = __ldg(reinterpret_cast<const uint32_t *>(spins_in + (size_t)PS[4 * g + q] * np + 4 * c));
            y |= (v & ~(v >> 1) & 0x01010101u) << q;   // bit 0 of each byte set and bit 1 clear: +1
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) w4[j] |= ((((y >> (8 * j)) & 0xFu) * 0x00204081u) & 0x01010101u) << g;
    }
}

__device__ __forceinline__ void msc_unpack_rows(const uint32_t (&w4)[4], int8_t *spins_out, int slot0, int np, int n,
                                                int c) {
    uint32_t real = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) real |= (4 * c + j < n ? 0xFFu : 0u) << (8 * j);
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        uint32_t e = 0u;   // byte q, bit j: replica 4g + q at position 4c + j
#pragma unroll
        for (int j = 0; j < 4; ++j) e |= ((w4[j] >> g) & 0x01010101u) << j;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t d = (((e >> (8 * q)) & 0xFu) * 0x00204081u) & 0x01010101u;
            *reinterpret_cast<uint32_t *>(spins_out + (size_t)(slot0 + 4 * g + q) * np + 4 * c) = ~(d * 0xFEu) & real;
        }
    }
}

// Philox4x32-10 for the eight counters (c0, c1_g, c2, c3) of one item, which
// differ only in word 1: the products of rounds 1-3 whose inputs do not depend
// on c1 are computed once (the result is identical to philox10 of each counter).
struct PhiloxShared {
    uint32_t u1;      // round 1: hi(M1 c2) ^ k0        (uniform)
    uint32_t l1;      // round 1: lo(M1 c2)              (uniform)
    uint32_t a, b;    // round 1: hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)
    uint32_t s0, s1;  // round 2: hi(M1 a) ^ l1 ^ k0', lo(M1 a)
    uint32_t h3, l3;  // round 3: hi(M0 s0), lo(M0 s0)
};

__device__ __forceinline__ PhiloxShared philox_shared(uint32_t c0, uint32_t c2, uint32_t c3, uint32_t k0,
                                                      uint32_t k1) {
    PhiloxShared p;
    uint32_t hi;
    mul_wide(0xCD9E8D57u, c2, p.l1, hi);
    p.u1 = hi ^ k0;
    mul_wide(0xD2511F53u, c0, p.b, hi);
    p.a = hi ^ c3 ^ k1;
    mul_wide(0xCD9E8D57u, p.a, p.s1, hi);
    p.s0 = hi ^ p.l1 ^ (k0 + 0x9E3779B9u);
    mul_wide(0xD2511F53u, p.s0, p.l3, p.h3);
    return p;
}

// Energy bookkeeping of the multi-spin-coded kernels. With |m| <= 31
// (NPL <= 5) every item adds, per replica 4g + q, 32 + m for an accepted flip
// and 32 for a rejected attempt into byte q of the lane's word ebias[g]; four
// items stay below 256 in every byte. After at most four items per lane the
// warp flushes: the 16-bit halves of the words are summed over the 32 lanes
// (at most 32 * 252 < 2^16, so no half carries into the next), the bias of 32
// per item is removed and lane r adds twice the result, the energy change of
// replica r, to Eacc[r]. This replaces one divergent shared atomic per accepted
// flip by branch-free byte arithmetic; the sums are exact integers, so the
// energies are the same as with per-flip updates. Wider counters (|m| up to
// 127) keep the per-flip atomics.
template <int NPL>
struct MscPackedE {
    static constexpr bool value = NPL <= 5;
};

// Pair decision table of the packed-energy items: entry (m0 + H/2) + H (m1 + H/2)
// holds E(m0) in its low and E(m1) in its high 16-bit lane, H = 2^(NPL+1)
// (|m| < H/2). One load decides two replicas; the byte offset of the entry
// is one dot product of the item's index bytes 4(m + H/2) with (1, H).
template <int NPL>
struct MscPairTab {
    static constexpr int H = 2 << NPL;
    static constexpr int words = MscPackedE<NPL>::value ? H * H : 0;
};

__host__ __device__ inline int msc_pair_words(int mmax) {
    return mmax <= 7 ? 256 : mmax <= 15 ? 1024 : mmax <= 31 ? 4096 : 0;
}

template <int NPL>
__device__ __forceinline__ void msc_fill_pair_table(uint32_t *PT, const uint32_t *T256, int tid, int NT) {
    constexpr int H = MscPairTab<NPL>::H;
    for (int i = tid; i < MscPairTab<NPL>::words; i += NT)
        PT[i] = (T256[i % H - H / 2 + 32] & 0xFFFFu) | (T256[i / H - H / 2 + 32] & 0xFFFF0000u);
}

__device__ __forceinline__ void msc_flush_energy(uint32_t (&ebias)[8], int &cnt, int32_t *Eacc, int lane) {
    const int nwarp = (int)__reduce_add_sync(0xFFFFFFFFu, (uint32_t)cnt);
    uint32_t mine = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const uint32_t slo = __reduce_add_sync(0xFFFFFFFFu, ebias[g] & 0x00FF00FFu);          // bytes 0, 2
        const uint32_t shi = __reduce_add_sync(0xFFFFFFFFu, (ebias[g] >> 8) & 0x00FF00FFu);   // bytes 1, 3
        if ((lane >> 2) == g) mine = (lane & 1) ? shi : slo;
        ebias[g] = 0u;
    }
    const int dm = (int)((lane & 2) ? (mine >> 16) : (mine & 0xFFFFu)) - 32 * nwarp;
    if (dm) atomicAdd(&Eacc[lane], 2 * dm);
    cnt = 0;
}

// Philox4x32-10 of two counters of one item (word 1 = c1a, c1b), finished
// from the shared round-1-3 products and advanced round by round together,
// so that the two dependency chains interleave. The round keys come
// precomputed in the kernel arguments (rk0[r] = key0 + r * 0x9E3779B9,
// rk1[r] = key1 + r * 0xBB67AE85), so they are operands, not additions. Round 1: only word 0 depends
// on c1. Round 2: the word-2 product (s0, s1) is shared, the word-0 product
// is per counter. Round 3: the word-0 product (h3, l3) is shared.
__device__ __forceinline__ void philox_from_shared2(const PhiloxShared &p, uint32_t c1a, uint32_t c1b,
                                                    const uint32_t (&rk0)[10], const uint32_t (&rk1)[10], uint4 &ra,
                                                    uint4 &rb) {
    uint32_t lo, hi, lo2, hi2;
    mul_wide(0xD2511F53u, p.u1 ^ c1a, lo, hi);
    mul_wide(0xD2511F53u, p.u1 ^ c1b, lo2, hi2);
    uint4 a = make_uint4(p.s0, p.s1, hi ^ p.b ^ rk1[1], lo);
    uint4 b = make_uint4(p.s0, p.s1, hi2 ^ p.b ^ rk1[1], lo2);
    mul_wide(0xCD9E8D57u, a.z, lo, hi);
    mul_wide(0xCD9E8D57u, b.z, lo2, hi2);
    a = make_uint4(hi ^ a.y ^ rk0[2], lo, p.h3 ^ a.w ^ rk1[2], p.l3);
    b = make_uint4(hi2 ^ b.y ^ rk0[2], lo2, p.h3 ^ b.w ^ rk1[2], p.l3);
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        uint32_t alo0, ahi0, alo1, ahi1, blo0, bhi0, blo1, bhi1;
        mul_wide(0xD2511F53u, a.x, alo0, ahi0);
        mul_wide(0xD2511F53u, b.x, blo0, bhi0);
        mul_wide(0xCD9E8D57u, a.z, alo1, ahi1);
        mul_wide(0xCD9E8D57u, b.z, blo1, bhi1);
        a = make_uint4(ahi1 ^ a.y ^ rk0[r], alo1, ahi0 ^ a.w ^ rk1[r], alo0);
        b = make_uint4(bhi1 ^ b.y ^ rk0[r], blo1, bhi0 ^ b.w ^ rk1[r], blo0);
    }
    ra = a;
    rb = b;
}

// One (position, word) item of a multi-spin-coded sweep: counts the frustrated
// bonds of the 32 replicas, decides the 32 attempts and records the energy
// change of every accepted flip, either in the lane's packed counters ebias
// (MscPackedE) or by a shared atomic on Eacc (local or a cluster peer's shared
// memory). Returns the mask of accepted replicas.
// Adds four bonds to the bit-sliced counters pl (one counter per replica):
// bit r of d_j = x ^ w_j is 1 iff bond j contributes +1 to m_r. Carry-save
// adders: d0 + d1 = s01 + 2 c01, d0 + .. + d3 = s + 2 (c01 + c23 + cs).
template <int NPL>
__device__ __forceinline__ void msc_csa4(uint32_t (&pl)[NPL], uint32_t x, uint32_t w0, uint32_t w1, uint32_t w2,
                                         uint32_t w3) {
    const uint32_t s01 = w0 ^ w1, c01 = (x ^ w0) & (x ^ w1);
    const uint32_t s23 = w2 ^ w3, c23 = (x ^ w2) & (x ^ w3);
    const uint32_t s = s01 ^ s23, cs = s01 & s23;
    const uint32_t t = pl[0] & s;
    pl[0] ^= s;
    const uint32_t u1 = pl[1] ^ c01 ^ c23, k1 = (pl[1] & c01) | (c23 & (pl[1] | c01));
    const uint32_t k2 = (u1 & cs) | (t & (u1 | cs));
    pl[1] = u1 ^ cs ^ t;
    uint32_t k = (pl[2] & k1) | (k2 & (pl[2] | k1));
    pl[2] ^= k1 ^ k2;
#pragma unroll
    for (int b = 3; b < NPL; ++b) {
        const uint32_t carry = pl[b] & k;
        pl[b] ^= k;
        k = carry;
    }
}

// Adds four bonds to counters kept in complemented form A_b = plane_b ^ x,
// where the input words are the raw neighbour words w_j (= d_j ^ x). A full
// adder keeps the form: (a^x) ^ (p^x) ^ (q^x) = (a^p^q) ^ x and, majority
// being self-dual, maj(a^x, p^x, q^x) = maj(a, p, q) ^ x. So two full adders
// take w0..w3 into the ones plane, one more takes their carries into the twos
// plane, and half adders (a^p^x, ((a^x) & (p^x)) ^ x) ripple the single carry
// upwards: 7 + 2 (NPL - 3) three-input logic ops per four bonds.
template <int NPL>
__device__ __forceinline__ void msc_step4x(uint32_t (&A)[NPL], uint32_t x, uint32_t w0, uint32_t w1, uint32_t w2,
                                           uint32_t w3) {
    const uint32_t c1 = (A[0] & w0) | (w1 & (A[0] | w0));
    A[0] ^= w0 ^ w1;
    const uint32_t c2 = (A[0] & w2) | (w3 & (A[0] | w2));
    A[0] ^= w2 ^ w3;
    uint32_t c = (A[1] & c1) | (c2 & (A[1] | c1));
    A[1] ^= c1 ^ c2;
#pragma unroll
    for (int b = 2; b < NPL; ++b) {
        const uint32_t nc = b + 1 < NPL ? (((A[b] ^ x) & (c ^ x)) ^ x) : 0u;
        A[b] ^= c ^ x;
        c = nc;
    }
}

// Delta swap of the bits selected by M between x >> s and y; zx, zy say that
// x or y is known to be zero (then the swap is a mask and a shift).
__device__ __forceinline__ void msc_swap(uint32_t &x, uint32_t &y, int s, uint32_t M, bool zx, bool zy) {
    if (zx && zy) return;
    if (zy) {
        y = (x >> s) & M;
        x &= ~(M << s);
    } else if (zx) {
        x = (y & M) << s;
        y &= ~M;
    } else {
        const uint32_t t = ((x >> s) ^ y) & M;
        x ^= t << s;
        y ^= t;
    }
}

template <int NPL, bool WEIGHTED>
__device__ __forceinline__ uint32_t msc_item(const SweepArgs &a, const uint32_t *Wsm, const uint32_t *T256, int p,
                                             uint32_t x, uint32_t c3, int blk, int32_t *Eacc,
                                             uint32_t (&ebias)[8], uint32_t &tent) {
    const uint32_t vid = __ldg(&a.g.vid[p]);
    uint32_t pl[NPL];
#pragma unroll
    for (int b = 0; b < NPL; ++b) pl[b] = 0u;
    uint32_t deg;
    if (a.g.mcol) {
        // Rows padded to whole 4-bond steps, entries = byte offsets of the
        // neighbours' words: one 8-byte load per step, no single-bond tail.
        const uint32_t h0 = __ldg(&a.g.mrp[p]), h1 = __ldg(&a.g.mrp[p + 1]);
        deg = h0 & 0xFFu;
        const unsigned char *Wb = reinterpret_cast<const unsigned char *>(Wsm);
        // The planes in complemented form (msc_step4x). With NPL = 3 (degree <= 7,
        // at most two steps) the plain adders starting from zero fold further
        // and stay cheaper.
        uint32_t A[NPL];
#pragma unroll
        for (int b = 0; b < NPL; ++b) A[b] = NPL >= 4 ? x : 0u;
        for (uint32_t q = h0 >> 8; q < (h1 >> 8); ++q) {
            const uint2 v = __ldg(&a.g.mcol[q]);
            const uint32_t o[4] = {v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16};
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                w[j] = *reinterpret_cast<const uint32_t *>(Wb + (WEIGHTED ? (o[j] & ~3u) : o[j]));
                if (WEIGHTED && (o[j] & 1u)) w[j] = ~w[j];
            }
            if (NPL >= 4) msc_step4x<NPL>(A, x, w[0], w[1], w[2], w[3]);
            else msc_csa4<NPL>(A, x, w[0], w[1], w[2], w[3]);
        }
#pragma unroll
        for (int b = 0; b < NPL; ++b) pl[b] = NPL >= 4 ? A[b] ^ x : A[b];
    } else {
        const uint32_t e0 = __ldg(&a.g.rp[p]), e1 = __ldg(&a.g.rp[p + 1]);
        deg = e1 - e0;
        uint32_t e = e0;
        for (; e + 4 <= e1; e += 4) {   // four bonds per step through carry-save adders
            uint32_t w0 = Wsm[__ldg(&a.g.col[e])], w1 = Wsm[__ldg(&a.g.col[e + 1])];
            uint32_t w2 = Wsm[__ldg(&a.g.col[e + 2])], w3 = Wsm[__ldg(&a.g.col[e + 3])];
            if (WEIGHTED) {
                if (__ldg(&a.g.wt[e]) < 0) w0 = ~w0;
                if (__ldg(&a.g.wt[e + 1]) < 0) w1 = ~w1;
                if (__ldg(&a.g.wt[e + 2]) < 0) w2 = ~w2;
                if (__ldg(&a.g.wt[e + 3]) < 0) w3 = ~w3;
            }
            msc_csa4<NPL>(pl, x, w0, w1, w2, w3);
        }
        for (; e < e1; ++e) {
            uint32_t d = x ^ Wsm[__ldg(&a.g.col[e])];
            if (WEIGHTED && __ldg(&a.g.wt[e]) < 0) d = ~d;
#pragma unroll
            for (int b = 0; b < NPL; ++b) {   // ripple-carry add of one bit per replica
                const uint32_t carry = pl[b] & d;
                pl[b] ^= d;
                d = carry;
            }
        }
    }
    constexpr bool PK = MscPackedE<NPL>::value;
    constexpr uint32_t H = (uint32_t)MscPairTab<NPL>::H;
    const uint32_t base = PK ? 2u * H - 4u * deg : 128u - deg;   // mb byte = 4(m + H/2) (PK) or m + 128
    // Both Philox calls of the item (slots 32 blk .. +15 and +16 .. +31).
    uint4 u0, u1;
    philox_from_shared2(philox_shared(vid, (uint32_t)a.k, c3, a.key0, a.key1), 2u * blk, 2u * blk + 1u, a.rk0, a.rk1,
                        u0, u1);
    // Byte q of r[g] = c of replica 4g + q: an 8 x 8 bit transpose in every byte lane.
    // Planes NPL..7 are zero, so a swap with a known-zero partner is a mask and
    // a shift (msc_swap); the zero set after each stage follows from NPL alone.
    uint32_t r[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) r[b] = b < NPL ? pl[b] : 0u;
#pragma unroll
    for (int b = 0; b < 4; ++b) msc_swap(r[b], r[b + 4], 4, 0x0F0F0F0Fu, b >= NPL, b + 4 >= NPL);
#pragma unroll
    for (int b = 0; b < 8; b += (b & 1) ? 3 : 1)   // 0, 1, 4, 5
        msc_swap(r[b], r[b + 2], 2, 0x33333333u, (b & 3) >= NPL, ((b + 2) & 3) >= NPL);
#pragma unroll
    for (int b = 0; b < 8; b += 2)
        msc_swap(r[b], r[b + 1], 1, 0x55555555u, (b & 3) >= NPL && ((b ^ 2) & 3) >= NPL,
                 ((b + 1) & 3) >= NPL && (((b + 1) ^ 2) & 3) >= NPL);
    uint32_t acc32 = 0, acct32 = 0;   // accepted; accepted or tied
    const uint32_t mq0 = (32u - deg) * 0x01010101u;   // 2c + 32 - deg = m + 32 per byte (PK)
    const unsigned char *tb = reinterpret_cast<const unsigned char *>(T256);
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const uint32_t mb = r[g] * (PK ? 8u : 2u) + base * 0x01010101u;
        const uint4 &uq = g < 4 ? u0 : u1;
        const uint32_t uw = (g & 3) == 0 ? uq.x : (g & 3) == 1 ? uq.y : (g & 3) == 2 ? uq.z : uq.w;
        uint32_t e01, e23;
        if (PK) {   // byte offsets of the pair entries: b0 + H b1 and b2 + H b3 of the bytes b = 4(m + H/2)
            e01 = *reinterpret_cast<const uint32_t *>(tb + __dp4a(mb, 0x00000001u | (H << 8), 0u));
            e23 = *reinterpret_cast<const uint32_t *>(tb + __dp4a(mb, 0x00010000u | (H << 24), 0u));
        } else {
            uint32_t e[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                e[q] = *reinterpret_cast<const uint32_t *>(tb + 4u * ((mb >> (8 * q)) & 0xFFu));
            e01 = __byte_perm(e[0], e[1], 0x5410u);
            e23 = __byte_perm(e[2], e[3], 0x5410u);
        }
        const uint32_t slo = __byte_perm(uw, 0u, 0x4140u) * 128u + e01;
        const uint32_t shi = __byte_perm(uw, 0u, 0x4342u) * 128u + e23;
        const uint32_t RT = prmt_sign(slo, shi, 0xFDB9u);                               // reject or tie
        const uint32_t RS = prmt_sign(slo - 0x00010001u, shi - 0x00010001u, 0xFDB9u);   // reject
        const uint32_t M = 0x01010101u << g;
        acc32 |= ~RT & M;
        acct32 |= ~RS & M;
        if (PK) {
            ebias[g] += ((r[g] * 2u + mq0) & ~RT) | (0x20202020u & RT);   // byte q: accepted ? 32 + m : 32
        } else if (~RT & 0x80808080u) {   // energy change 2m = 2(mb byte - 128) of each accepted replica
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (!((RT >> (8 * q)) & 1u)) atomicAdd(&Eacc[4 * g + q], 2 * ((int)((mb >> (8 * q)) & 0xFFu) - 128));
        }
    }
    uint32_t tie = acct32 & ~acc32;
    tent = 0u;
    if (tie) {   // the low 24 bits of the uniform decide: the item's first tie is queued for
                 // the warp (msc_queue_tie), further ties of the same item are settled here
        const uint32_t *tab = a.tables + (size_t)a.tidx[a.k] * (a.g.mmax + 1);
        bool first = true;
        do {
            const int bit = __ffs(tie) - 1;
            tie &= tie - 1u;
            const int g = bit & 7;
            uint32_t rg = r[0];   // count byte of the replica at this bit: byte bit >> 3 of r[bit & 7]
#pragma unroll
            for (int j = 1; j < 8; ++j)
                if (g == j) rg = r[j];
            const int m = 2 * (int)((rg >> (bit & 24)) & 0xFFu) - (int)deg;
            if (first) {   // the item's first tie goes to the warp's queue
                tent = 0x80000000u | (uint32_t)p << 13 | (uint32_t)bit << 8 | (uint32_t)m;
                first = false;
                continue;
            }
            const uint32_t T = __ldg(&tab[m]);
            const int rep = 4 * (bit & 7) + (bit >> 3);
            if (sweep_tail_bits(vid, 32u * blk + rep, (uint32_t)a.k, c3, a.key0, a.key1) < (T & 0xFFFFFFu)) {
                acc32 |= 1u << bit;
                atomicAdd(&Eacc[rep], 2 * m);
            }
        } while (tie);
    }
    return acc32;
}

// Ties queued by the items of a warp (entry = flag | p << 13 | bit << 8 | m)
// are settled together: each lane takes one entry, draws the low 24 bits of
// its uniform and applies an accepted flip to the word (and its copy in the
// peer CTA), the energy and the accept count. Items of one colour class never
// read each other's words, so a flip applied after the other items of the
// class is the same as one applied at once; every queue is emptied before the
// class barrier.
__device__ __forceinline__ void msc_drain_ties(const SweepArgs &a, const uint32_t *TQ, int qc, uint32_t *Wsm,
                                               uint32_t *Wpeer, int32_t *Eacc, int blk, uint32_t c3, uint32_t vmask,
                                               uint32_t &nacc, int lane) {
    __syncwarp();
    const uint32_t *tab = a.tables + (size_t)a.tidx[a.k] * (a.g.mmax + 1);
    for (int i = lane; i < qc; i += 32) {
        const uint32_t e = TQ[i];
        const int p = (int)((e >> 13) & 0xFFFFu), bit = (int)((e >> 8) & 31u), m = (int)(e & 0xFFu);
        const int rep = 4 * (bit & 7) + (bit >> 3);
        const uint32_t T = __ldg(&tab[m]);
        if (sweep_tail_bits(__ldg(&a.g.vid[p]), 32u * blk + rep, (uint32_t)a.k, c3, a.key0, a.key1) <
            (T & 0xFFFFFFu)) {
            atomicXor(&Wsm[p], 1u << bit);
            if (Wpeer) atomicXor(&Wpeer[p], 1u << bit);
            atomicAdd(&Eacc[rep], 2 * m);
            nacc += (vmask >> bit) & 1u;
        }
    }
    __syncwarp();
}

// Appends the lanes' queue entries (tent != 0) to the warp's tie queue; drains
// it once it holds more than 32 entries (capacity 64).
__device__ __forceinline__ void msc_queue_tie(const SweepArgs &a, uint32_t *TQ, int &qc, uint32_t tent, uint32_t *Wsm,
                                              uint32_t *Wpeer, int32_t *Eacc, int blk, uint32_t c3, uint32_t vmask,
                                              uint32_t &nacc, int lane) {
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, tent != 0u);
    if (bal) {
        if (tent) TQ[qc + __popc(bal & ((1u << lane) - 1u))] = tent;
        qc += __popc(bal);
        if (qc > 32) {
            msc_drain_ties(a, TQ, qc, Wsm, Wpeer, Eacc, blk, c3, vmask, nacc, lane);
            qc = 0;
        }
    }
}

template <int NPL, bool WEIGHTED, int NTB, int MINB>
__global__ void __launch_bounds__(NTB, MINB) k_sweep_msc(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const bool act = !a.active || a.active[a.k];
    const int nsweeps = act ? a.S : 0;
    const int np = a.g.np, n = a.g.n;
    uint32_t *T256 = reinterpret_cast<uint32_t *>(smem);          // [256] decision table (see above)
    uint32_t *PT = T256 + 256;                                      // [H * H] pair table (packed energies)
    uint32_t *Wsm = PT + MscPairTab<NPL>::words;                    // [np]
    int32_t *cls = reinterpret_cast<int32_t *>(Wsm + np);
    const int csz = (a.g.ncol + 1 + 3) & ~3;
    int32_t *Eacc = cls + csz;      // [32]
    int32_t *PS = Eacc + 32;        // [32]
    int32_t *misc = PS + 32;        // best E, step, sweep, slot, copy-from (r+1), changed
    uint32_t *TQ = reinterpret_cast<uint32_t *>(misc + 8) + (threadIdx.x >> 5) * 64;   // [warps][64] tie queues

    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    const uint32_t *tab = a.tables + (size_t)a.tidx[a.k] * (a.g.mmax + 1);
    for (int i = tid; i < 256; i += NT) T256[i] = msc_entry(i, MscPackedE<NPL>::value, tab, a.g.mmax);
    if (MscPackedE<NPL>::value) {
        __syncthreads();
        msc_fill_pair_table<NPL>(PT, T256, tid, NT);
    }
    for (int i = tid; i <= a.g.ncol; i += NT) cls[i] = a.g.cls[i];

    for (int lb = blockIdx.x; lb < a.nblk; lb += gridDim.x) {
        const int blk = a.blk_base + lb;
        const int slot0 = blk * 32;
        if (tid < 32) PS[tid] = act ? a.parent[slot0 + tid] : slot0 + tid;
        if (tid == 0) {
            const int4 br = a.best_rec[blk];
            misc[0] = br.x; misc[1] = br.y; misc[2] = br.z; misc[3] = br.w;
            misc[4] = 0; misc[5] = 0;
        }
        __syncthreads();
        if (tid < 32) Eacc[tid] = a.E_in[PS[tid]];
        // Load: 32 int8 spin rows -> one bit word per position.
        for (int c = tid; c < (np >> 2); c += NT) {
            uint32_t w4[4];
            msc_pack_rows(a.spins_in, PS, np, c, w4);
#pragma unroll
            for (int j = 0; j < 4; ++j) Wsm[4 * c + j] = w4[j];
        }
        __syncthreads();
        uint32_t vmask = 0u;   // bits of the live replicas
        for (int r = 0; r < 32; ++r) vmask |= (slot0 + r < a.R ? 1u : 0u) << msc_bit(r);
        uint32_t nacc = 0;
        uint32_t ebias[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        int cnt = 0;
        for (int s = 0; s < nsweeps; ++s) {
            const uint32_t c3 = TAG_SWEEP | (uint32_t)s;
            for (int c = 0; c < a.g.ncol; ++c) {
                const int p0 = cls[c], p1 = cls[c + 1];
                const int nr = (p1 - p0 + NT - 1) / NT;   // rounds of the class, uniform over the CTA
                int qc = 0;   // entries in this warp's tie queue
                for (int rd = 0; rd < nr; ++rd) {
                    const int p = p0 + tid + rd * NT;
                    uint32_t tent = 0u;
                    if (p < p1) {
                        const uint32_t x = Wsm[p];
                        const uint32_t acc32 =
                            msc_item<NPL, WEIGHTED>(a, Wsm, MscPackedE<NPL>::value ? PT : T256, p, x, c3, blk, Eacc,
                                                    ebias, tent);
                        if (acc32) {
                            Wsm[p] = x ^ acc32;
                            nacc += __popc(acc32 & vmask);
                        }
                        ++cnt;
                    }
                    msc_queue_tie(a, TQ, qc, tent, Wsm, nullptr, Eacc, blk, c3, vmask, nacc, lane);
                    if (MscPackedE<NPL>::value && ((rd & 3) == 3 || rd == nr - 1))
                        msc_flush_energy(ebias, cnt, Eacc, lane);
                }
                if (qc) msc_drain_ties(a, TQ, qc, Wsm, nullptr, Eacc, blk, c3, vmask, nacc, lane);
                __syncthreads();
            }
            if (tid == 0) {
                int bq = -1, bE = 0x7FFFFFFF;
                for (int q = 0; q < 32; ++q)
                    if (slot0 + q < a.R && Eacc[q] < bE) { bE = Eacc[q]; bq = q; }
                misc[4] = 0;
                if (bq >= 0) {
                    atomicMin(&a.sweep_emin[(size_t)a.k * a.S + s], bE);
                    if (bE < misc[0]) {
                        misc[0] = bE; misc[1] = a.k; misc[2] = s; misc[3] = slot0 + bq;
                        misc[4] = bq + 1; misc[5] = 1;
                    }
                }
            }
            __syncthreads();
            if (misc[4]) {
                const int rq = misc[4] - 1;
                uint32_t *dst = reinterpret_cast<uint32_t *>(a.best_cfg + (size_t)blk * np);
                for (int c = tid; c < (np >> 2); c += NT) {
                    uint32_t v = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool real = 4 * c + j < n;
                        v |= (real ? (((Wsm[4 * c + j] >> msc_bit(rq)) & 1u) ? 0x01u : 0xFFu) : 0u) << (8 * j);
                    }
                    dst[c] = v;
                }
                __syncthreads();
            }
        }
        // Store: bit words -> int8 spin rows (fields are not kept by this layout).
        for (int c = tid; c < (np >> 2); c += NT) {
            uint32_t w4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) w4[j] = Wsm[4 * c + j];
            msc_unpack_rows(w4, a.spins_out, slot0, np, n, c);
        }
        if (tid < 32) a.E_out[slot0 + tid] = Eacc[tid];
        if (tid == 0 && misc[5]) a.best_rec[blk] = make_int4(misc[0], misc[1], misc[2], misc[3]);
        const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, nacc);
        if (act && lane == 0 && wsum) atomicAdd(&a.accepts[a.k], (unsigned long long)wsum);
        __syncthreads();
    }
}

// Multi-spin coding with a thread-block cluster of two CTAs per word. Both
// CTAs keep a full copy of the word array; inside a colour class CTA r takes
// the items at even (r = 0) or odd (r = 1) offsets, and every changed word is
// stored into both copies (the peer's through distributed shared memory). A
// cluster barrier closes each class. The 32 energies live in CTA 0, which
// also does the best tracking; CTA 1 adds its energy changes there remotely.
// Halving the work unit lets the SMs balance 2 x words CTAs dynamically.
template <int NPL, bool WEIGHTED>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 4) k_sweep_msc_pair(const SweepArgs a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    extern __shared__ __align__(16) unsigned char smem[];
    const bool act = !a.active || a.active[a.k];
    const int nsweeps = act ? a.S : 0;
    const int np = a.g.np, n = a.g.n;
    uint32_t *T256 = reinterpret_cast<uint32_t *>(smem);          // [256] decision table (see above)
    uint32_t *PT = T256 + 256;                                      // [H * H] pair table (packed energies)
    uint32_t *Wsm = PT + MscPairTab<NPL>::words;                    // [np]
    int32_t *cls = reinterpret_cast<int32_t *>(Wsm + np);
    const int csz = (a.g.ncol + 1 + 3) & ~3;
    int32_t *Eacc = cls + csz;      // [32] (used in CTA 0)
    int32_t *PS = Eacc + 32;        // [32]
    int32_t *misc = PS + 32;        // best E, step, sweep, slot, copy-from (r+1), changed
    uint32_t *Wpeer = cluster.map_shared_rank(Wsm, rank ^ 1);
    int32_t *E0 = cluster.map_shared_rank(Eacc, 0);
    uint32_t *TQ = reinterpret_cast<uint32_t *>(misc + 8) + (threadIdx.x >> 5) * 64;   // [warps][64] tie queues

    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    const uint32_t *tab = a.tables + (size_t)a.tidx[a.k] * (a.g.mmax + 1);
    for (int i = tid; i < 256; i += NT) T256[i] = msc_entry(i, MscPackedE<NPL>::value, tab, a.g.mmax);
    if (MscPackedE<NPL>::value) {
        __syncthreads();
        msc_fill_pair_table<NPL>(PT, T256, tid, NT);
    }
    for (int i = tid; i <= a.g.ncol; i += NT) cls[i] = a.g.cls[i];

    const int ncl = (int)(gridDim.x >> 1);
    for (int lb = (int)(blockIdx.x >> 1); lb < a.nblk; lb += ncl) {   // uniform within the cluster
        const int blk = a.blk_base + lb;
        const int slot0 = blk * 32;
        if (tid < 32) PS[tid] = act ? a.parent[slot0 + tid] : slot0 + tid;
        if (tid == 0) {
            const int4 br = a.best_rec[blk];
            misc[0] = br.x; misc[1] = br.y; misc[2] = br.z; misc[3] = br.w;
            misc[4] = 0; misc[5] = 0;
        }
        __syncthreads();
        if (tid < 32 && rank == 0) Eacc[tid] = a.E_in[PS[tid]];
        for (int c = tid; c < (np >> 2); c += NT) {
            uint32_t w4[4];
            msc_pack_rows(a.spins_in, PS, np, c, w4);
#pragma unroll
            for (int j = 0; j < 4; ++j) Wsm[4 * c + j] = w4[j];
        }
        cluster.sync();   // both copies loaded, energies in place
        uint32_t vmask = 0u;   // bits of the live replicas
        for (int r = 0; r < 32; ++r) vmask |= (slot0 + r < a.R ? 1u : 0u) << msc_bit(r);
        uint32_t nacc = 0;
        uint32_t ebias[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        int cnt = 0;
        for (int s = 0; s < nsweeps; ++s) {
            const uint32_t c3 = TAG_SWEEP | (uint32_t)s;
            for (int c = 0; c < a.g.ncol; ++c) {
                const int p0 = cls[c], p1 = cls[c + 1];
                const int nr = (p1 - p0 + 2 * NT - 1) / (2 * NT);   // rounds, uniform over the cluster
                int qc = 0;   // entries in this warp's tie queue
                for (int rd = 0; rd < nr; ++rd) {
                    const int p = p0 + 2 * tid + rank + rd * 2 * NT;
                    uint32_t tent = 0u;
                    if (p < p1) {
                        const uint32_t x = Wsm[p];
                        const uint32_t acc32 = msc_item<NPL, WEIGHTED>(a, Wsm, MscPackedE<NPL>::value ? PT : T256, p, x, c3,
                                                                       blk, E0, ebias, tent);
                        if (acc32) {
                            Wsm[p] = x ^ acc32;
                            Wpeer[p] = x ^ acc32;
                            nacc += __popc(acc32 & vmask);
                        }
                        ++cnt;
                    }
                    msc_queue_tie(a, TQ, qc, tent, Wsm, Wpeer, E0, blk, c3, vmask, nacc, lane);
                    if (MscPackedE<NPL>::value && ((rd & 3) == 3 || rd == nr - 1))
                        msc_flush_energy(ebias, cnt, E0, lane);
                }
                if (qc) msc_drain_ties(a, TQ, qc, Wsm, Wpeer, E0, blk, c3, vmask, nacc, lane);
                cluster.sync();
            }
            if (rank == 0 && tid == 0) {
                int bq = -1, bE = 0x7FFFFFFF;
                for (int q = 0; q < 32; ++q)
                    if (slot0 + q < a.R && Eacc[q] < bE) { bE = Eacc[q]; bq = q; }
                misc[4] = 0;
                if (bq >= 0) {
                    atomicMin(&a.sweep_emin[(size_t)a.k * a.S + s], bE);
                    if (bE < misc[0]) {
                        misc[0] = bE; misc[1] = a.k; misc[2] = s; misc[3] = slot0 + bq;
                        misc[4] = bq + 1; misc[5] = 1;
                    }
                }
            }
            __syncthreads();
            if (misc[4]) {   // CTA 0 only (CTA 1 never sets it)
                const int rq = misc[4] - 1;
                uint32_t *dst = reinterpret_cast<uint32_t *>(a.best_cfg + (size_t)blk * np);
                for (int c = tid; c < (np >> 2); c += NT) {
                    uint32_t v = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool real = 4 * c + j < n;
                        v |= (real ? (((Wsm[4 * c + j] >> msc_bit(rq)) & 1u) ? 0x01u : 0xFFu) : 0u) << (8 * j);
                    }
                    dst[c] = v;
                }
            }
            cluster.sync();   // the copy reads CTA 0's words before the next sweep changes them
        }
        // Store: each CTA writes half of the columns from its own (complete) copy.
        for (int c = 2 * tid + rank; c < (np >> 2); c += 2 * NT) {
            uint32_t w4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) w4[j] = Wsm[4 * c + j];
            msc_unpack_rows(w4, a.spins_out, slot0, np, n, c);
        }
        if (rank == 0) {
            if (tid < 32) a.E_out[slot0 + tid] = Eacc[tid];
            if (tid == 0 && misc[5]) a.best_rec[blk] = make_int4(misc[0], misc[1], misc[2], misc[3]);
        }
        const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, nacc);
        if (act && lane == 0 && wsum) atomicAdd(&a.accepts[a.k], (unsigned long long)wsum);
        cluster.sync();   // neither copy is reused before both CTAs are done with this word
    }
}

template <bool W>
void *msc_pair_kernel(int mmax) {
    if (mmax <= 7) return reinterpret_cast<void *>(&k_sweep_msc_pair<3, W>);
    if (mmax <= 15) return reinterpret_cast<void *>(&k_sweep_msc_pair<4, W>);
    if (mmax <= 31) return reinterpret_cast<void *>(&k_sweep_msc_pair<5, W>);
    if (mmax <= 63) return reinterpret_cast<void *>(&k_sweep_msc_pair<6, W>);
    return reinterpret_cast<void *>(&k_sweep_msc_pair<7, W>);
}

template <bool W>
void *msc_kernel(int mmax) {
    if (mmax <= 7) return reinterpret_cast<void *>(&k_sweep_msc<3, W, 256, 4>);
    if (mmax <= 15) return reinterpret_cast<void *>(&k_sweep_msc<4, W, 256, 4>);
    if (mmax <= 31) return reinterpret_cast<void *>(&k_sweep_msc<5, W, 256, 4>);
    if (mmax <= 63) return reinterpret_cast<void *>(&k_sweep_msc<6, W, 256, 4>);
    return reinterpret_cast<void *>(&k_sweep_msc<7, W, 256, 4>);   // c <= 127: mb = 2c + 128 - deg stays in a byte
}

template <bool W>
void *packed_kernel(int threads) {
    switch (threads) {
        // 64 registers a thread (at least 1024 threads per SM): the packed item
        // with its lane decisions spills at 40 registers.
        case 128: return reinterpret_cast<void *>(&k_sweep_packed<W, 128, 8>);
        case 256: return reinterpret_cast<void *>(&k_sweep_packed<W, 256, 4>);
        case 384: return reinterpret_cast<void *>(&k_sweep_packed<W, 384, 2>);
        case 512: return reinterpret_cast<void *>(&k_sweep_packed<W, 512, 2>);
        default: return reinterpret_cast<void *>(&k_sweep_packed<W, 1024, 1>);
    }
}

template <int G, int FB, bool W>
void *kernel_ptr() {
    return reinterpret_cast<void *>(&k_sweep<G, FB, W>);
}

void *select_kernel(int G, int fb, bool weighted, int threads, int mmax) {
    if (fb == 1) return weighted ? msc_kernel<true>(mmax) : msc_kernel<false>(mmax);
    if (fb == 2) return weighted ? msc_pair_kernel<true>(mmax) : msc_pair_kernel<false>(mmax);
    if (fb == 7) return weighted ? packed_kernel<true>(threads) : packed_kernel<false>(threads);
    if (G == 1) {
        if (fb == 16) return weighted ? kernel_ptr<1, 16, true>() : kernel_ptr<1, 16, false>();
        return weighted ? kernel_ptr<1, 8, true>() : kernel_ptr<1, 8, false>();
    }
    if (fb == 16) return weighted ? kernel_ptr<2, 16, true>() : kernel_ptr<2, 16, false>();
    return weighted ? kernel_ptr<2, 8, true>() : kernel_ptr<2, 8, false>();
}

}  // namespace

size_t sweep_smem_bytes(const GraphDev &g, int G, int field_bits, int threads) {
    if (field_bits == 1 || field_bits == 2)   // multi-spin coded: 32 replicas per word (2: CTA pairs)
        return (size_t)g.np * 4 + (256 + (size_t)msc_pair_words(g.mmax)) * 4 + (size_t)((g.ncol + 1 + 3) & ~3) * 4 +
               (32 + 32 + 8) * 4 +
               (size_t)(threads / 32) * 64 * 4;   // tie queues
    if (field_bits == 7)
        return (size_t)(g.np + 32) * 4 + 256 * 4 + (size_t)((g.ncol + 1 + 3) & ~3) * 4 + 16 * 4 +
               (size_t)((((g.np + 31) / 32) + 1) & ~1) * 4 + (size_t)(threads / 32) * PK_QCAP * 8;
    const int HW = field_bits == 16 ? 2 : 1;
    return (size_t)g.np * G * 4 * (1 + HW) + (size_t)((g.mmax + 1 + 3) & ~3) * 4 +
           (size_t)((g.ncol + 1 + 3) & ~3) * 4 + (size_t)(8 * G + 8) * 4;
}

cudaError_t sweep_configure(const GraphDev &g, int R, int G, int field_bits, int threads,
                            bool weighted, SweepConfig *cfg) {
    if (field_bits == 1 || field_bits == 2) {
        G = 8;
        threads = 256;
    } else if (field_bits == 7) {
        G = 1;
    }
    const size_t smem = sweep_smem_bytes(g, G, field_bits, threads);
    void *fn = select_kernel(G, field_bits, weighted, threads, g.mmax);
    // The attribute belongs to the kernel function, not to a context: only ever
    // raise it, so that contexts configured earlier keep launching.
    {
        static std::mutex mu;
        static std::unordered_map<void *, size_t> raised;
        std::lock_guard<std::mutex> lock(mu);
        size_t &cur = raised[fn];
        if (smem > cur) {
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            cur = smem;
        }
    }
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nblk = (R + 4 * G - 1) / (4 * G);
    if (field_bits == 2) {
        // One cluster of two CTAs per word; the hardware schedules them as slots free up.
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(2 * nblk);
        lc.blockDim = dim3(threads);
        lc.dynamicSmemBytes = smem;
        int ncl = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, fn, &lc);
        if (e != cudaSuccess) return e;
        if (ncl < 1) return cudaErrorInvalidConfiguration;
        cfg->G = G;
        cfg->field_bits = field_bits;
        cfg->threads = threads;
        cfg->smem = smem;
        cfg->grid = 2 * nblk;
        return cudaSuccess;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    cfg->G = G;
    cfg->field_bits = field_bits;
    cfg->threads = threads;
    cfg->smem = smem;
    cfg->grid = nblk < occ * sms ? nblk : occ * sms;
    return cudaSuccess;
}

cudaError_t launch_sweep(const SweepConfig &cfg, const SweepArgs &a, cudaStream_t st) {
    void *fn = select_kernel(cfg.G, cfg.field_bits, a.g.wt != nullptr, cfg.threads, a.g.mmax);
    void *args[] = {const_cast<SweepArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3(cfg.grid), dim3(cfg.threads), args, cfg.smem, st);
}

}  // namespace pa
