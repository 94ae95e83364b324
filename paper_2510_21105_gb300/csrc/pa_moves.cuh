// pa_moves.cuh -- non-local (Houdayer) moves and ESS-adaptive temperature
// steps (internal to libpa.so).
#pragma once

#include "pa_internal.cuh"

namespace pa {

// Houdayer cluster move of step k (Sec. 3 names "periodic non-local moves";
// this is the library's reading): slots are paired by sorting
// (Philox word (r>>2, 0, k, tag 2)[r&3], r); for pair m = (a, b) the set
// D = {i : x^a_i != x^b_i}, the seed is the (u_m mod |D|)-th element of D in
// ascending vertex order with u_m = Philox word (m>>2, 1, k, tag 2)[m&3], the
// cluster C is the seed's connected component in the graph induced on D,
// and both replicas flip on C (E_a + E_b is unchanged).
struct NlmArgs {
    GraphDev g;
    const int32_t *pos;            // [n] position of each vertex
    int8_t *spins;                 // population after the sweeps of step k
    int16_t *fields;               // rebuilt after a move; null when the sweep layout keeps no fields
    int32_t *E;
    int32_t R, k;
    uint32_t key0, key1;
    const int32_t *active;         // [K] or nullptr
    int32_t *pairs;                // [K] moves performed (block moves: accepted)
    unsigned long long *flips;     // [K] summed cluster (block) sizes
    int32_t kind;                  // 0 Houdayer pairs, 1 block moves
    int32_t block;                 // block moves: size b
    const double *qrow;            // block moves: q = exp(-2 beta) per table row
    const int32_t *tidx;           // [K] table row of step k
};
// Block move of step k (alternative reading of the non-local moves): every
// slot r flips B = the first b vertices of a breadth-first search from
// vertex (Philox word (r>>2, 2, k, tag 2)[r&3] mod n), rows scanned in CSR
// order, iff m <= 0 or u < A(m): m = -sum over edges (i in B, j not in B)
// of w x_i x_j, u = Philox word (r>>2, 3, k, tag 2)[r&3],
// A(m) = min(2^32-1, floor(2^32 q^m)), q^m by square and multiply.
size_t nlm_scratch_bytes(int32_t R);
size_t nlm_smem_bytes(int32_t np);
size_t nlm_block_smem_bytes(int32_t np, int32_t block);
// Enqueues the move; *launches receives the number of kernels launched.
cudaError_t launch_nonlocal(const NlmArgs &a, void *scratch, cudaStream_t st, int *launches);

// ESS-adaptive step (Sec. 3 names "adaptive control of stochasticity"; this
// is the library's reading): beta lives on the grid n * delta with
// delta = dbeta_max / 2^J. From grid index n_prev, level j proposes
// dn_j = min(2^(J-j), nmax - n_prev); the weights q_j^{E_r - E_min} with
// q_j = exp(-dn_j delta) give ESS_j = A_j^2 / B_j (A, B the pairwise-tree sums
// of w and w*w); the smallest j with ESS_j >= rho R is taken, else J.
struct AdaptArgs {
    const int32_t *E;
    const int32_t *emin;           // [K] minimum of the step (computed first)
    int32_t R, k, J, nmax, nch;
    double rhoR, delta;
    const double *qpow;            // [2^J][32]: row dn-1 = squarings of exp(-dn delta)
    double *part;                  // [J+1][2][nch] chunk tree sums of w and w*w
    int32_t *state;                // [0] = n_prev, [1] = current level (mode 2)
    int32_t *qsel, *active, *tidx, *jsel;
    double *beta;
    int32_t mode;                  // 1 ESS rule, 2 acceptance-rate rule
    const unsigned long long *accepts;   // [K] accepted flips per step (mode 2)
    double acc_lo_n, acc_hi_n;     // mode 2: band edges times n R S (attempts per step)
};
// Acceptance-rate rule (mode 2, an alternative reading): the level starts at
// j = 0; a previous step that accepted fewer than acc_lo n R S flips moves j
// one level finer (j + 1, at most J), more than acc_hi n R S one level
// coarser (j - 1, at least 0); dn = min(2^(J-j), nmax - n_prev).
cudaError_t launch_adapt(const AdaptArgs &a, cudaStream_t st);

// Stagnation reheating (an alternative reading of the adaptive control):
// at the start of step k > 0 the lowest sweep-end energy of step k-1 updates
// the running best; reheat_after consecutive steps without a lower one move
// the schedule index back by reheat_back (not below 0) and restart the
// count, otherwise the index advances by one (at most K-1). The step's
// resampling uses qpow row i when the index advanced from i-1, else row K
// (q = 1, identity).
struct ReheatArgs {
    const int32_t *sweep_emin;     // [K][S]
    const double *betas;           // [K] schedule
    int32_t k, K, S, after, back;
    int32_t *state;                // [0] index, [1] steps without a new best, [2] best energy
    int32_t *tidx, *qsel, *isel;   // [K] table row, qpow row, schedule index
    double *beta;                  // [K] beta of step k
};
cudaError_t launch_reheat(const ReheatArgs &a, cudaStream_t st);

}  // namespace pa
