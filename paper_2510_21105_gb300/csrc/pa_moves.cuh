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
    int16_t *fields;
    int32_t *E;
    int32_t R, k;
    uint32_t key0, key1;
    const int32_t *active;         // [K] or nullptr
    int32_t *pairs;                // [K] moves performed
    unsigned long long *flips;     // [K] summed cluster sizes
};
size_t nlm_scratch_bytes(int32_t R);
size_t nlm_smem_bytes(int32_t np);
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
    int32_t *state;                // [0] = n_prev
    int32_t *qsel, *active, *tidx, *jsel;
    double *beta;
};
cudaError_t launch_adapt(const AdaptArgs &a, cudaStream_t st);

}  // namespace pa
