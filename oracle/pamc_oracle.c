/*
 * pamc_oracle.c -- plain, slow, single-threaded CPU oracle for Population
 * Annealing Monte Carlo (PAMC) on Max-Cut.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file. It shares no code, header,
 * table generator or helper with the CUDA library: it is an independent
 * statement of what the GPU path must compute, written for a reader to check
 * by eye. Integer state is exact; the only floating point is FP64 for the
 * acceptance thresholds, the resampling weights and the free-energy sum.
 *
 * Paper: "New Best-Known Max-Cut Solution for the G63 Instance in the G-Set
 * Benchmark" (arXiv 2510.21105).
 *   Eq. 1          Max-Cut objective: maximise 1/2 sum_{i<j} w_ij (1 - x_i x_j)
 *                  over x in {-1,+1}^N.
 *   Sec. 2         Max-Cut equals minimising an Ising energy whose couplings
 *                  are the negated edge weights (antiferromagnetic for w > 0),
 *                  i.e. E(x) = sum_{i<j} w_ij x_i x_j and cut = (W - E)/2.
 *   Sec. 3         The solver is Population Annealing Monte Carlo with
 *                  adaptive control of stochasticity and periodic non-local
 *                  moves, run on one GPU. The paper defines none of these
 *                  steps further (Sec. 4 defers the details). Every rule
 *                  below beyond Eq. 1 and the Ising mapping is therefore a
 *                  reading of the method; the readings are listed with the
 *                  design notes of the repository.
 *
 * Parity status. Each function is pinned by tests against mathematics, not
 * against itself:
 *   orc_philox4x32_10   cuRAND's host Philox4x32-10 generator (library routine)
 *   orc_greedy_colour   networkx greedy colouring in index order; classes are
 *                       independent sets; an even torus gives two colours
 *   orc_energy          direct count of cut edges (cut = (W - E)/2) and brute
 *                       force maxima for N <= 20
 *   orc_accept_table    monotone in m; chi-square of fixed-beta histograms
 *                       against the exact Boltzmann law (via orc_anneal)
 *   orc_resample        sum of copies = R, identity at dbeta = 0, mean copies
 *                       = R t_r / T over the offset
 *   orc_anneal          PA free-energy estimate against exact Z (N <= 12);
 *                       best cut <= and, on small graphs, = brute force;
 *                       final energies equal full recomputation
 *   orc_houdayer_pair   cluster = networkx connected component of the seed in
 *                       G[D]; E_a + E_b invariant
 *   orc_block_move      block = the first b vertices of a networkx BFS that
 *                       visits neighbours in row order; m = half the energy
 *                       change computed by full recomputation; brute-force
 *                       acceptance frequency against min(1, exp(-2 beta m))
 *   adaptive mode       chosen step meets ESS >= rho R unless it is the
 *                       finest; beta monotone and ends at beta_max
 *   adaptive = 2        level sequence recomputed from the recorded accepted
 *                       flips; beta monotone, ends at beta_max
 *   reheating           schedule index sequence recomputed from the recorded
 *                       sweep minima; non-advancing steps resample as the
 *                       identity
 * Parity against the paper itself is unpinned for every step the paper does
 * not define (Sec. 3-4): sweep order, acceptance rule, resampling scheme,
 * adaptive control (ESS rule, acceptance-rate rule, stagnation reheating)
 * and non-local moves (Houdayer pairs, block moves).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11). Ten rounds; each  */
/* round multiplies counter words 0 and 2 by the two Philox constants,      */
/* xors the high halves with the other counter words and the key, and the   */
/* key is advanced by the two Weyl constants between rounds.                */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream tags (top four bits of counter word 3). */
enum { TAG_SWEEP = 0, TAG_RESAMPLE = 1, TAG_NONLOCAL = 2, TAG_INIT = 3, TAG_TAIL = 4 };

/* One 32-bit random word: word `w` of Philox(key = seed, counter = c). */
static uint32_t rng_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                         uint32_t c3, int w)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[w];
}

/* ------------------------------------------------------------------------ */
/* Graph helpers. The CSR stores every undirected edge in both rows.         */
/* ------------------------------------------------------------------------ */
static int weight_of(const int8_t *w, int64_t e) { return w ? (int)w[e] : 1; }

/* Ising energy E(x) = sum over undirected edges (i<j) of w_ij x_i x_j
 * (Eq. 1 with the Sec. 2 mapping: cut(x) = (W - E(x)) / 2). */
int64_t orc_energy(int32_t n, const int64_t *rp, const int32_t *col, const int8_t *w,
                   const int8_t *x)
{
    int64_t E = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (j > i) E += (int64_t)weight_of(w, e) * x[i] * x[j];
        }
    return E;
}

/* W = sum over undirected edges of w_ij. */
int64_t orc_total_weight(int32_t n, const int64_t *rp, const int32_t *col, const int8_t *w)
{
    int64_t W = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (col[e] > i) W += weight_of(w, e);
    return W;
}

/* Local field h_i = sum_j w_ij x_j. */
static int32_t local_field(const int64_t *rp, const int32_t *col, const int8_t *w,
                           const int8_t *x, int32_t i)
{
    int32_t h = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) h += weight_of(w, e) * x[col[e]];
    return h;
}

/* First-fit greedy colouring in vertex-index order: vertex i takes the
 * smallest colour not used by any neighbour j < i. Returns the number of
 * colours. The sweep visits colour 0, 1, ..., C-1 and, within a colour,
 * vertices in ascending index. */
int32_t orc_greedy_colour(int32_t n, const int64_t *rp, const int32_t *col, int32_t *colour)
{
    int32_t ncol = 0;
    int32_t *seen = (int32_t *)calloc((size_t)n + 2, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (j < i) seen[colour[j]] = i + 1;
        }
        int32_t c = 0;
        while (seen[c] == i + 1) ++c;
        colour[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(seen);
    return ncol;
}

/* Metropolis acceptance thresholds for inverse temperature beta: a move that
 * raises the energy by dE = 2m (m >= 1) is accepted iff the 32-bit uniform
 * word u satisfies u < T[m], with T[m] = floor(2^32 exp(-beta * 2m)) clamped
 * to 2^32 - 1. Moves with m <= 0 are always accepted; T[0] is unused and set
 * to 2^32 - 1. */
void orc_accept_table(double beta, int32_t mmax, uint32_t *T)
{
    T[0] = 0xFFFFFFFFu;
    for (int32_t m = 1; m <= mmax; ++m) {
        double p = exp(-(beta * (double)(2 * m)));
        double v = floor(ldexp(p, 32));
        T[m] = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
    }
}

/* ------------------------------------------------------------------------ */
/* Resampling (population annealing reweighting, one temperature step).     */
/* ------------------------------------------------------------------------ */

/* q^d by right-to-left square and multiply over the bits of d, in FP64. */
static double power_sq_mul(double q, uint32_t d)
{
    double acc = 1.0, s = q;
    while (d) {
        if (d & 1u) acc = acc * s;
        d >>= 1;
        s = s * s;
    }
    return acc;
}

/* Pairwise tree sum over indices 0..R-1 padded with zeros to a power of
 * two: level by level, s_i <- s_{2i} + s_{2i+1}. */
static double tree_sum(const double *v, int32_t R)
{
    size_t L = 1;
    while (L < (size_t)R) L <<= 1;
    double *s = (double *)calloc(L, sizeof(double));
    memcpy(s, v, (size_t)R * sizeof(double));
    while (L > 1) {
        for (size_t i = 0; i < L / 2; ++i) s[i] = s[2 * i] + s[2 * i + 1];
        L /= 2;
    }
    double r = s[0];
    free(s);
    return r;
}

/* Cumulative copy count of systematic resampling: the number of the R
 * equally spaced points (with offset o / 2^32) that fall below cumulative
 * integer weight P out of total T:  floor((P R 2^32 + o T) / (T 2^32)). */
static int64_t systematic_count(uint64_t P, int32_t R, uint64_t T, uint32_t o)
{
    unsigned __int128 num = (unsigned __int128)P * (unsigned __int128)R;
    num = (num << 32) + (unsigned __int128)o * (unsigned __int128)T;
    unsigned __int128 den = (unsigned __int128)T << 32;
    return (int64_t)(num / den);
}

/* One resampling of a population of R replicas with energies E, given
 * q = exp(-dbeta) and the offset word o:
 *   E_min = min_r E_r, d_r = E_r - E_min, w_r = q^{d_r},
 *   A = tree sum of w_r, t_r = floor(2^32 w_r) (integer weights),
 *   T = sum t_r, P_r = sum_{s<r} t_s,
 *   parent r gets copies into new slots [F(P_r), F(P_r + t_r)).
 * Outputs: counts[r] (may be NULL), parent[s] for every new slot s (may be
 * NULL), E_min, A, T. Returns 0, or -1 if R < 1 or q is not in (0, 1]. */
/* One shard of a population split over ranks (for the sharded-resampling
 * tests): with the population's E_min given, the weights of the shard's n
 * slots, their pairwise tree sum (zero-padded to a power of two), the integer
 * weights t[n] and their total. Same arithmetic as orc_resample. */
void orc_shard_partials(int32_t n, const int32_t *E, int32_t emin, double q, double *A, uint64_t *T,
                        uint64_t *t)
{
    double *w = (double *)malloc((size_t)n * sizeof(double));
    uint64_t tot = 0;
    for (int32_t r = 0; r < n; ++r) {
        w[r] = power_sq_mul(q, (uint32_t)((int64_t)E[r] - emin));
        t[r] = (uint64_t)floor(ldexp(w[r], 32));
        tot += t[r];
    }
    *A = tree_sum(w, n);
    *T = tot;
    free(w);
}

/* Systematic resampling boundary F(P) (see orc_resample). */
int64_t orc_systematic_count(uint64_t P, int32_t R, uint64_t T, uint32_t o)
{
    return systematic_count(P, R, T, o);
}

int orc_resample(int32_t R, const int32_t *E, double q, uint32_t o,
                 int32_t *counts, int32_t *parent,
                 int32_t *emin_out, double *A_out, uint64_t *T_out)
{
    if (R < 1 || !(q > 0.0) || !(q <= 1.0)) return -1;
    int32_t emin = E[0];
    for (int32_t r = 1; r < R; ++r) if (E[r] < emin) emin = E[r];
    double *w = (double *)malloc((size_t)R * sizeof(double));
    uint64_t *t = (uint64_t *)malloc((size_t)R * sizeof(uint64_t));
    uint64_t T = 0;
    for (int32_t r = 0; r < R; ++r) {
        w[r] = power_sq_mul(q, (uint32_t)((int64_t)E[r] - emin));
        t[r] = (uint64_t)floor(ldexp(w[r], 32));
        T += t[r];
    }
    double A = tree_sum(w, R);
    uint64_t P = 0;
    int32_t filled = 0;
    for (int32_t r = 0; r < R; ++r) {
        int64_t lo = systematic_count(P, R, T, o);
        int64_t hi = systematic_count(P + t[r], R, T, o);
        int32_t n_r = (int32_t)(hi - lo);
        if (counts) counts[r] = n_r;
        if (parent)
            for (int64_t s = lo; s < hi; ++s) parent[s] = r;
        filled += n_r;
        P += t[r];
    }
    free(w);
    free(t);
    if (emin_out) *emin_out = emin;
    if (A_out) *A_out = A;
    if (T_out) *T_out = T;
    return filled == R ? 0 : -2;
}

/* ------------------------------------------------------------------------ */
/* Houdayer cluster move between two replicas a and b at the same beta.     */
/* D = {i : x^a_i != x^b_i}; the seed is the (u mod |D|)-th element of D in  */
/* ascending index; C = the connected component of the seed in the graph    */
/* induced on D (edges of either sign); both replicas flip on C. Returns    */
/* |C| (0 if D is empty). cluster (may be NULL) receives a 0/1 mask.         */
/* ------------------------------------------------------------------------ */
int32_t orc_houdayer_pair(int32_t n, const int64_t *rp, const int32_t *col,
                          int8_t *xa, int8_t *xb, uint32_t u, uint8_t *cluster)
{
    int32_t nd = 0;
    for (int32_t i = 0; i < n; ++i) nd += xa[i] != xb[i];
    if (n < 1) return 0;
    if (cluster) memset(cluster, 0, (size_t)n);
    if (nd == 0) return 0;
    int32_t target = (int32_t)(u % (uint32_t)nd), seedv = -1;
    for (int32_t i = 0, c = 0; i < n; ++i)
        if (xa[i] != xb[i]) {
            if (c == target) { seedv = i; break; }
            ++c;
        }
    uint8_t *in = (uint8_t *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t head = 0, tail = 0;
    in[seedv] = 1;
    queue[tail++] = seedv;
    while (head < tail) {
        int32_t i = queue[head++];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (!in[j] && xa[j] != xb[j]) { in[j] = 1; queue[tail++] = j; }
        }
    }
    for (int32_t h = 0; h < tail; ++h) {
        int32_t i = queue[h];
        xa[i] = (int8_t)-xa[i];
        xb[i] = (int8_t)-xb[i];
        if (cluster) cluster[i] = 1;
    }
    free(in);
    free(queue);
    return tail;
}

/* Pairing for the non-local move of step k: slots sorted by the key
 * (word r&3 of Philox(counter = (r>>2, 0, k, tag 2)), r); pairs are
 * consecutive entries of the sorted order. */
typedef struct { uint32_t key; int32_t slot; } pair_key;

static int cmp_pair_key(const void *pa, const void *pb)
{
    const pair_key *a = (const pair_key *)pa, *b = (const pair_key *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->slot > b->slot) - (a->slot < b->slot);
}

void orc_nlm_order(int32_t R, uint64_t seed, int32_t k, int32_t *order)
{
    pair_key *pk = (pair_key *)malloc((size_t)R * sizeof(pair_key));
    for (int32_t r = 0; r < R; ++r) {
        pk[r].key = rng_word(seed, (uint32_t)r >> 2, 0, (uint32_t)k,
                             (uint32_t)TAG_NONLOCAL << 28, r & 3);
        pk[r].slot = r;
    }
    qsort(pk, (size_t)R, sizeof(pair_key), cmp_pair_key);
    for (int32_t r = 0; r < R; ++r) order[r] = pk[r].slot;
    free(pk);
}

static uint32_t nlm_seed_word(uint64_t seed, int32_t k, int32_t m)
{
    return rng_word(seed, (uint32_t)m >> 2, 1, (uint32_t)k, (uint32_t)TAG_NONLOCAL << 28, m & 3);
}

/* ------------------------------------------------------------------------ */
/* Block move (alternative reading of the non-local moves, nlm_kind = 1):    */
/* one replica flips a connected block of up to b spins as a single         */
/* Metropolis move.                                                          */
/*   B    the first b vertices reached by breadth-first search from the      */
/*        seed vertex, each row scanned in CSR order (fewer when the seed's  */
/*        component is smaller);                                             */
/*   m    half the energy change of flipping B: only the edges leaving B     */
/*        change sign, so m = -sum_{i in B, j not in B} w_ij x_i x_j;        */
/*   rule accept iff m <= 0 or u < A(m), A(m) = min(2^32 - 1,                */
/*        floor(2^32 q^m)) with q = exp(-2 beta) and q^m by square and       */
/*        multiply (the same power as the resampling weights).              */
/* Returns |B| if the move is accepted (x flipped on B, *E += 2m), else 0.   */
/* block (may be NULL) receives the 0/1 mask of B either way.               */
/* ------------------------------------------------------------------------ */
int32_t orc_block_move(int32_t n, const int64_t *rp, const int32_t *col, const int8_t *w,
                       int8_t *x, int32_t *E, int32_t b, double q, int32_t seedv, uint32_t u,
                       uint8_t *block)
{
    if (n < 1 || b < 1 || seedv < 0 || seedv >= n) return 0;
    uint8_t *in = (uint8_t *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t head = 0, tail = 0;
    in[seedv] = 1;
    queue[tail++] = seedv;
    while (head < tail && tail < b) {
        int32_t i = queue[head++];
        for (int64_t e = rp[i]; e < rp[i + 1] && tail < b; ++e) {
            int32_t j = col[e];
            if (!in[j]) { in[j] = 1; queue[tail++] = j; }
        }
    }
    int64_t leaving = 0;                 /* sum over edges leaving B of w x_i x_j */
    for (int32_t h = 0; h < tail; ++h) {
        int32_t i = queue[h];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (!in[j]) leaving += (int64_t)(w ? w[e] : 1) * x[i] * x[j];
        }
    }
    int64_t m = -leaving;
    int accept = m <= 0;
    if (!accept) {
        double v = floor(ldexp(power_sq_mul(q, (uint32_t)m), 32));
        uint32_t A = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
        accept = u < A;
    }
    if (block) for (int32_t i = 0; i < n; ++i) block[i] = in[i];
    if (accept) {
        for (int32_t h = 0; h < tail; ++h) x[queue[h]] = (int8_t)-x[queue[h]];
        *E += (int32_t)(2 * m);
    }
    free(in);
    free(queue);
    return accept ? tail : 0;
}

/* Random words of the block move of slot r at step k: the seed vertex is
 * word r&3 of Philox((r>>2, 2, k, tag 2)) mod n and the acceptance word is
 * word r&3 of Philox((r>>2, 3, k, tag 2)). */
static int32_t block_seed_vertex(uint64_t seed, int32_t k, int32_t r, int32_t n)
{
    return (int32_t)(rng_word(seed, (uint32_t)r >> 2, 2, (uint32_t)k, (uint32_t)TAG_NONLOCAL << 28, r & 3) %
                     (uint32_t)n);
}

static uint32_t block_accept_word(uint64_t seed, int32_t k, int32_t r)
{
    return rng_word(seed, (uint32_t)r >> 2, 3, (uint32_t)k, (uint32_t)TAG_NONLOCAL << 28, r & 3);
}

/* ------------------------------------------------------------------------ */
/* Full anneal.                                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t nlm_period;       /* non-local move after the sweeps of step k when
                                 k > 0 and k % nlm_period == 0; 0 = off */
    int32_t adaptive;         /* 0: betas[] is the schedule; 1: ESS-adaptive;
                                 2: acceptance-rate-adaptive */
    double rho;               /* adaptive: ESS / R threshold */
    int32_t adapt_J;          /* adaptive: finest grid level J */
    double adapt_dbeta_max;   /* adaptive: coarsest step */
    double beta_max;          /* adaptive: final inverse temperature */
    int32_t nlm_kind;         /* 0: Houdayer pair moves; 1: block moves */
    int32_t nlm_block;        /* block moves: block size b >= 1 */
    double acc_lo, acc_hi;    /* adaptive = 2: acceptance-rate band */
    int32_t reheat_after;     /* fixed schedules: reheat after this many steps
                                 without a new best energy; 0 = off */
    int32_t reheat_back;      /* schedule entries a reheat steps back */
} orc_opts;

typedef struct {              /* every pointer may be NULL */
    int8_t *spins;            /* [R][n] final population, vertex order */
    int32_t *E;               /* [R] final energies */
    double *step_beta;        /* [K] beta used by the sweeps of step k */
    int32_t *step_emin;       /* [K] E_min of the resampling at step k */
    double *step_A;           /* [K] weight sum A of step k */
    uint64_t *step_T;         /* [K] integer weight total T of step k */
    uint32_t *step_o;         /* [K] systematic offset word of step k */
    int64_t *step_accepts;    /* [K] accepted flips in the sweeps of step k */
    double *step_lnZ;         /* [K] free-energy estimate ln Z(beta_k) */
    int32_t *step_counts;     /* [K][R] copy counts of step k */
    int32_t *step_sweep_emin; /* [K][S] min energy over replicas after each sweep */
    int32_t *step_nlm_pairs;  /* [K] pairs with a non-empty D (block moves:
                                 accepted moves) */
    int64_t *step_nlm_flips;  /* [K] sum of cluster sizes (block moves: spins
                                 flipped by accepted moves) */
    int32_t *step_jsel;       /* [K] adaptive: chosen grid level; reheating:
                                 schedule index used by step k */
    int8_t *best_config;      /* [n] configuration of the best energy */
    int32_t best[4];          /* best energy, step, sweep, slot (-1 if none) */
    int32_t steps_run;
} orc_out;

typedef struct {
    int32_t n;
    const int64_t *rp;
    const int32_t *col;
    const int8_t *w;
    int32_t ncol;
    int32_t *class_start;     /* [ncol+1] */
    int32_t *class_list;      /* [n] vertices grouped by colour, ascending */
    int32_t maxdeg;
} graph_view;

static int build_view(graph_view *g, int32_t n, const int64_t *rp, const int32_t *col,
                      const int8_t *w)
{
    g->n = n; g->rp = rp; g->col = col; g->w = w;
    int32_t *colour = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    g->ncol = n > 0 ? orc_greedy_colour(n, rp, col, colour) : 0;
    g->class_start = (int32_t *)calloc((size_t)g->ncol + 1, sizeof(int32_t));
    g->class_list = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) g->class_start[colour[i] + 1]++;
    for (int32_t c = 0; c < g->ncol; ++c) g->class_start[c + 1] += g->class_start[c];
    int32_t *fill = (int32_t *)calloc((size_t)g->ncol + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        int32_t c = colour[i];
        g->class_list[g->class_start[c] + fill[c]++] = i;
    }
    g->maxdeg = 0;
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] - rp[i] > g->maxdeg) g->maxdeg = (int32_t)(rp[i + 1] - rp[i]);
    free(fill);
    free(colour);
    return 0;
}

static void free_view(graph_view *g)
{
    free(g->class_start);
    free(g->class_list);
}

/* The 32-bit uniform of a Metropolis attempt on vertex i of replica `slot`
 * at step k, sweep s. Its top 8 bits are byte (slot mod 4) of word
 * (floor(slot/4) mod 4) of Philox(i, floor(slot/16), k, s), so one Philox
 * call serves 16 replicas; its low 24 bits are the top 24 bits of word
 * (slot mod 4) of Philox(i, floor(slot/4), k, tag 4 | s). Both are uniform
 * and independent, so u is uniform on [0, 2^32). A comparison u < T needs
 * the low 24 bits only when the top byte of u equals that of T. */
static uint32_t sweep_uniform(uint64_t seed, int32_t i, int32_t slot, int32_t k, int32_t s)
{
    uint32_t word = rng_word(seed, (uint32_t)i, (uint32_t)slot >> 4, (uint32_t)k,
                             ((uint32_t)TAG_SWEEP << 28) | (uint32_t)s, (slot >> 2) & 3);
    uint32_t top = (word >> (8 * (slot & 3))) & 0xFFu;
    uint32_t tail = rng_word(seed, (uint32_t)i, (uint32_t)slot >> 2, (uint32_t)k,
                             ((uint32_t)TAG_TAIL << 28) | (uint32_t)s, slot & 3);
    return (top << 24) | (tail >> 8);
}

/* Threads of the timing build (OpenMP); 1 in the checking build. */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(int32_t want)
{
    if (want > 0) omp_set_num_threads(want);
    return omp_get_max_threads();
}
#else
int orc_threads(int32_t want)
{
    (void)want;
    return 1;
}
#endif

/* Uniforms of n attempts (vertex i[t], replica slot[t]) at step k, sweep s,
 * for the tests. */
void orc_sweep_uniforms(uint64_t seed, int32_t n, const int32_t *i, const int32_t *slot, int32_t k,
                        int32_t s, uint32_t *u)
{
    for (int32_t t = 0; t < n; ++t) u[t] = sweep_uniform(seed, i[t], slot[t], k, s);
}

/* One Metropolis sweep of replica `slot` at step k, sweep index s: colours in
 * order, vertices ascending within a colour. The field h_i is recomputed
 * from the neighbours at every visit. Returns the number of accepted flips
 * and adds the energy change to *E. */
static int64_t sweep_replica(const graph_view *g, int8_t *x, int32_t *E, const uint32_t *T,
                             uint64_t seed, int32_t slot, int32_t k, int32_t s)
{
    int64_t acc = 0;
    for (int32_t c = 0; c < g->ncol; ++c)
        for (int32_t idx = g->class_start[c]; idx < g->class_start[c + 1]; ++idx) {
            int32_t i = g->class_list[idx];
            int32_t h = local_field(g->rp, g->col, g->w, x, i);
            int32_t m = -x[i] * h;            /* dE = 2m for flipping x_i */
            int accept = m <= 0;
            if (!accept) accept = sweep_uniform(seed, i, slot, k, s) < T[m];
            if (accept) {
                x[i] = (int8_t)-x[i];
                *E += 2 * m;
                ++acc;
            }
        }
    return acc;
}

/* Initial population: i.i.d. uniform spins (exact equilibrium at beta = 0);
 * spin i of slot r is +1 iff bit 31 of word r&3 of
 * Philox(counter = (i, r>>2, 0, tag 3)) is set. */
static void init_population(const graph_view *g, int8_t *pop, int32_t *E, int32_t R, uint64_t seed)
{
    for (int32_t r = 0; r < R; ++r) {
        int8_t *x = pop + (size_t)r * g->n;
        for (int32_t i = 0; i < g->n; ++i) {
            uint32_t u = rng_word(seed, (uint32_t)i, (uint32_t)r >> 2, 0,
                                  (uint32_t)TAG_INIT << 28, r & 3);
            x[i] = (u >> 31) ? 1 : -1;
        }
        E[r] = (int32_t)orc_energy(g->n, g->rp, g->col, g->w, x);
    }
}

/* Copy replicas according to parent[] (new slot s <- old slot parent[s]). */
static void apply_parents(int8_t *pop, int8_t *tmp, int32_t *E, int32_t *Etmp,
                          const int32_t *parent, int32_t R, int32_t n)
{
    memcpy(tmp, pop, (size_t)R * n);
    memcpy(Etmp, E, (size_t)R * sizeof(int32_t));
    for (int32_t s = 0; s < R; ++s) {
        memcpy(pop + (size_t)s * n, tmp + (size_t)parent[s] * n, (size_t)n);
        E[s] = Etmp[parent[s]];
    }
}

/* Non-local moves of step k over the whole population. */
static void nonlocal_moves(const graph_view *g, int8_t *pop, int32_t *E, int32_t R, uint64_t seed,
                           int32_t k, int32_t *pairs_out, int64_t *flips_out)
{
    int32_t *order = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    orc_nlm_order(R, seed, k, order);
    int32_t pairs = 0;
    int64_t flips = 0;
    for (int32_t m = 0; 2 * m + 1 < R; ++m) {
        int32_t a = order[2 * m], b = order[2 * m + 1];
        int8_t *xa = pop + (size_t)a * g->n, *xb = pop + (size_t)b * g->n;
        int32_t csize = orc_houdayer_pair(g->n, g->rp, g->col, xa, xb,
                                          nlm_seed_word(seed, k, m), NULL);
        if (csize > 0) {
            ++pairs;
            flips += csize;
            E[a] = (int32_t)orc_energy(g->n, g->rp, g->col, g->w, xa);
            E[b] = (int32_t)orc_energy(g->n, g->rp, g->col, g->w, xb);
        }
    }
    free(order);
    if (pairs_out) *pairs_out = pairs;
    if (flips_out) *flips_out = flips;
}

/* Block moves of step k: every slot independently (see orc_block_move). */
static void block_moves(const graph_view *g, int8_t *pop, int32_t *E, int32_t R, uint64_t seed,
                        int32_t k, int32_t b, double beta_k, int32_t *moves_out, int64_t *flips_out)
{
    const double q = exp(-2.0 * beta_k);
    int32_t moves = 0;
    int64_t flips = 0;
    for (int32_t r = 0; r < R; ++r) {
        int32_t size = orc_block_move(g->n, g->rp, g->col, g->w, pop + (size_t)r * g->n, &E[r], b, q,
                                      block_seed_vertex(seed, k, r, g->n), block_accept_word(seed, k, r),
                                      NULL);
        if (size > 0) { ++moves; flips += size; }
    }
    if (moves_out) *moves_out = moves;
    if (flips_out) *flips_out = flips;
}

/* Adaptive step choice (reading of "adaptive control of stochasticity"):
 * beta moves on the grid beta = n * delta, delta = dbeta_max / 2^J. From
 * the current grid index n_prev, level j proposes dn_j = 2^(J-j) (clamped
 * to n_max - n_prev). For each j, w = q_j^{d_r} with q_j = exp(-dn_j delta),
 * ESS_j = A_j^2 / B_j with A_j, B_j the tree sums of w and w*w. The chosen
 * level is the smallest j with ESS_j >= rho R, else J. Returns dn. */
static int32_t adaptive_choose(const int32_t *E, int32_t R, int32_t n_prev, int32_t n_max,
                               int32_t J, double delta, double rhoR, int32_t *jsel)
{
    int32_t emin = E[0];
    for (int32_t r = 1; r < R; ++r) if (E[r] < emin) emin = E[r];
    double *w = (double *)malloc((size_t)R * sizeof(double));
    double *w2 = (double *)malloc((size_t)R * sizeof(double));
    int32_t chosen = J, dn_chosen = 0;
    for (int32_t j = 0; j <= J; ++j) {
        int32_t dn = 1 << (J - j);
        if (dn > n_max - n_prev) dn = n_max - n_prev;
        double q = exp(-((double)dn * delta));
        for (int32_t r = 0; r < R; ++r) {
            w[r] = power_sq_mul(q, (uint32_t)((int64_t)E[r] - emin));
            w2[r] = w[r] * w[r];
        }
        double A = tree_sum(w, R), B = tree_sum(w2, R);
        double ess = (A * A) / B;
        dn_chosen = dn;
        if (ess >= rhoR) { chosen = j; break; }
    }
    free(w);
    free(w2);
    *jsel = chosen;
    return dn_chosen;
}

/* Run PAMC. Schedule: step k (0..K-1) resamples the population from beta_{k-1}
 * to beta_k (beta_{-1} = 0), runs S sweeps at beta_k with best tracking after
 * every sweep, then applies the non-local move when due. In adaptive mode K
 * is the maximum number of steps and betas may be NULL.
 * Best tracking: after each sweep, replicas are scanned in slot order and
 * a strictly lower energy replaces the best, so ties go to the earliest
 * (step, sweep) and then the lowest slot.
 * Returns 0 on success, -1 on invalid arguments. */
int orc_anneal(int32_t n, const int64_t *rp, const int32_t *col, const int8_t *w,
               const double *betas, int32_t K, int32_t R, int32_t S, uint64_t seed,
               const orc_opts *opts, orc_out *out)
{
    if (n < 1 || K < 0 || R < 1 || S < 0) return -1;
    orc_opts o = {0, 0, 0.0, 0, 0.0, 0.0, 0, 1, 0.0, 1.0, 0, 0};
    if (opts) o = *opts;
    if (o.nlm_kind < 0 || o.nlm_kind > 1 || (o.nlm_kind == 1 && o.nlm_block < 1)) return -1;
    if (o.reheat_after < 0 || (o.reheat_after > 0 && (o.adaptive || o.reheat_back < 1))) return -1;
    if (!o.adaptive) {
        double prev = 0.0;
        for (int32_t k = 0; k < K; ++k) {
            if (!isfinite(betas[k]) || betas[k] < prev) return -1;
            prev = betas[k];
        }
    } else if (o.adaptive < 0 || o.adaptive > 2 || o.adapt_J < 0 || o.adapt_J > 20 ||
               !(o.adapt_dbeta_max > 0.0) || !(o.beta_max >= 0.0) || !isfinite(o.beta_max) ||
               (o.adaptive == 2 && !(o.acc_lo >= 0.0 && o.acc_lo <= o.acc_hi && o.acc_hi <= 1.0))) {
        return -1;
    }
    graph_view g;
    build_view(&g, n, rp, col, w);
    int8_t *pop = (int8_t *)malloc((size_t)R * n);
    int8_t *tmp = (int8_t *)malloc((size_t)R * n);
    int32_t *E = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    int32_t *Etmp = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    int32_t *parent = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    int32_t *counts = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    uint32_t *T = (uint32_t *)malloc((size_t)(g.maxdeg + 1) * sizeof(uint32_t));
    init_population(&g, pop, E, R, seed);

    double delta = o.adaptive ? ldexp(o.adapt_dbeta_max, -o.adapt_J) : 0.0;
    int32_t n_max = o.adaptive ? (int32_t)floor(o.beta_max / delta + 0.5) : 0;
    double rhoR = o.rho * (double)R;
    int32_t n_prev = 0;
    int32_t j_prev = 0;                 /* adaptive = 2: current level */
    int64_t acc_prev = 0;               /* accepted flips of the previous step */
    int32_t i_prev = 0, stall = 0;      /* reheating: schedule index, steps without a new best */
    int32_t best_run = 0x7FFFFFFF, step_min = 0x7FFFFFFF;
    const double attempts = (double)((int64_t)n * R * S);

    double beta_prev = 0.0;
    double lnZ = (double)n * log(2.0);
    int32_t best_E = 0x7FFFFFFF, best_k = -1, best_s = -1, best_r = -1;
    int32_t k;
    for (k = 0; k < K; ++k) {
        double beta_k, q;
        if (o.adaptive) {
            if (n_prev >= n_max) break;
            int32_t jsel, dn;
            if (o.adaptive == 2) {
                /* Acceptance-rate control (alternative reading of the adaptive
                 * stochasticity): a previous step that accepted fewer than
                 * acc_lo of its attempts refines the temperature step by one
                 * level (dn halves), more than acc_hi coarsens it by one. */
                if (k > 0) {
                    if ((double)acc_prev < o.acc_lo * attempts) {
                        if (j_prev < o.adapt_J) ++j_prev;
                    } else if ((double)acc_prev > o.acc_hi * attempts) {
                        if (j_prev > 0) --j_prev;
                    }
                }
                jsel = j_prev;
                dn = 1 << (o.adapt_J - j_prev);
                if (dn > n_max - n_prev) dn = n_max - n_prev;
            } else {
                dn = adaptive_choose(E, R, n_prev, n_max, o.adapt_J, delta, rhoR, &jsel);
            }
            if (out->step_jsel) out->step_jsel[k] = jsel;
            n_prev += dn;
            beta_k = (double)n_prev * delta;
            q = exp(-((double)dn * delta));
        } else if (o.reheat_after > 0) {
            /* Stagnation reheating (alternative reading of the adaptive
             * stochasticity): the schedule index advances by one per step
             * (and stays at the last entry) unless reheat_after consecutive
             * steps found no lower energy at their sweep ends; then it steps
             * back by reheat_back entries (not below 0) and the count
             * restarts. A step that does not advance the index leaves the
             * population unweighted (q = 1, identity resampling). */
            int32_t i = 0, forward = 1;
            if (k > 0) {
                if (step_min < best_run) { best_run = step_min; stall = 0; }
                else ++stall;
                if (stall >= o.reheat_after) {
                    i = i_prev - o.reheat_back < 0 ? 0 : i_prev - o.reheat_back;
                    stall = 0;
                } else {
                    i = i_prev + 1 < K ? i_prev + 1 : K - 1;
                }
                forward = i == i_prev + 1;
            }
            if (out->step_jsel) out->step_jsel[k] = i;
            beta_k = betas[i];
            q = forward ? exp(-(betas[i] - (i > 0 ? betas[i - 1] : 0.0))) : 1.0;
            i_prev = i;
        } else {
            beta_k = betas[k];
            q = exp(-(beta_k - beta_prev));
        }
        double dbeta = beta_k - beta_prev;
        uint32_t ow = rng_word(seed, 0, 0, (uint32_t)k, (uint32_t)TAG_RESAMPLE << 28, 0);
        int32_t emin;
        double A;
        uint64_t Tt;
        orc_resample(R, E, q, ow, counts, parent, &emin, &A, &Tt);
        apply_parents(pop, tmp, E, Etmp, parent, R, n);
        lnZ += -dbeta * (double)emin + log(A / (double)R);
        if (out->step_beta) out->step_beta[k] = beta_k;
        if (out->step_emin) out->step_emin[k] = emin;
        if (out->step_A) out->step_A[k] = A;
        if (out->step_T) out->step_T[k] = Tt;
        if (out->step_o) out->step_o[k] = ow;
        if (out->step_lnZ) out->step_lnZ[k] = lnZ;
        if (out->step_counts) memcpy(out->step_counts + (size_t)k * R, counts, (size_t)R * sizeof(int32_t));

        orc_accept_table(beta_k, g.maxdeg, T);
        int64_t acc = 0;
        step_min = 0x7FFFFFFF;
        for (int32_t s = 0; s < S; ++s) {
            int32_t sweep_min = 0x7FFFFFFF;
            /* Replicas are independent between resamplings, so the timing
             * build (-fopenmp) may sweep them on several threads; the result,
             * an integer sum and per-replica state, does not depend on it. */
#pragma omp parallel for reduction(+ : acc) schedule(dynamic, 4)
            for (int32_t r = 0; r < R; ++r)
                acc += sweep_replica(&g, pop + (size_t)r * n, &E[r], T, seed, r, k, s);
            for (int32_t r = 0; r < R; ++r) {
                if (E[r] < sweep_min) sweep_min = E[r];
                if (E[r] < best_E) {
                    best_E = E[r]; best_k = k; best_s = s; best_r = r;
                    if (out->best_config) memcpy(out->best_config, pop + (size_t)r * n, (size_t)n);
                }
            }
            if (out->step_sweep_emin) out->step_sweep_emin[(size_t)k * S + s] = sweep_min;
            if (sweep_min < step_min) step_min = sweep_min;
        }
        if (out->step_accepts) out->step_accepts[k] = acc;
        acc_prev = acc;

        int32_t pairs = 0;
        int64_t flips = 0;
        if (o.nlm_period > 0 && k > 0 && k % o.nlm_period == 0) {
            if (o.nlm_kind == 1)
                block_moves(&g, pop, E, R, seed, k, o.nlm_block, beta_k, &pairs, &flips);
            else
                nonlocal_moves(&g, pop, E, R, seed, k, &pairs, &flips);
        }
        if (out->step_nlm_pairs) out->step_nlm_pairs[k] = pairs;
        if (out->step_nlm_flips) out->step_nlm_flips[k] = flips;
        beta_prev = beta_k;
    }
    out->steps_run = k;
    out->best[0] = best_k >= 0 ? best_E : 0;
    out->best[1] = best_k;
    out->best[2] = best_s;
    out->best[3] = best_r;
    if (out->spins) memcpy(out->spins, pop, (size_t)R * n);
    if (out->E) memcpy(out->E, E, (size_t)R * sizeof(int32_t));
    free(pop); free(tmp); free(E); free(Etmp); free(parent); free(counts); free(T);
    free_view(&g);
    return 0;
}

/* Replay of one temperature step k on a given population (vertex order),
 * for a subset of the new slots: energies of the whole input population are
 * recomputed, the population is resampled from beta_prev to beta_k, each
 * listed slot takes its parent's configuration and runs S sweeps at beta_k,
 * and, when nlm_now is set, listed pairs of the step-k pairing get the
 * non-local move (nlm_block = 0) or every listed slot gets its block move of
 * size nlm_block (nlm_block >= 1). For pair moves the subset must contain
 * both members of every pair it touches. Outputs the listed slots' spins [nsub][n] and
 * energies, the accepted flips summed over the listed slots, and optionally
 * the copy counts [R]. Returns 0, -1 on invalid arguments, -3 if a pair is
 * split by the subset. */
int orc_step(int32_t n, const int64_t *rp, const int32_t *col, const int8_t *w,
             int32_t R, int32_t S, uint64_t seed, int32_t k, double beta_prev, double beta_k,
             int32_t nlm_now, int32_t nlm_block, const int8_t *spins_in, int32_t nsub,
             const int32_t *sub, int8_t *spins_out, int32_t *E_out, int32_t *counts,
             int64_t *accepts_out)
{
    if (n < 1 || R < 1 || S < 0 || !(beta_k >= beta_prev) || !isfinite(beta_k) || nlm_block < 0)
        return -1;
    graph_view g;
    build_view(&g, n, rp, col, w);
    int32_t *E = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    for (int32_t r = 0; r < R; ++r)
        E[r] = (int32_t)orc_energy(n, rp, col, w, spins_in + (size_t)r * n);
    int32_t *parent = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    uint32_t ow = rng_word(seed, 0, 0, (uint32_t)k, (uint32_t)TAG_RESAMPLE << 28, 0);
    orc_resample(R, E, exp(-(beta_k - beta_prev)), ow, counts, parent, NULL, NULL, NULL);
    uint32_t *T = (uint32_t *)malloc((size_t)(g.maxdeg + 1) * sizeof(uint32_t));
    orc_accept_table(beta_k, g.maxdeg, T);
    int64_t acc = 0;
    int rc = 0;
    for (int32_t q = 0; q < nsub; ++q) {
        int32_t s = sub[q];
        int8_t *x = spins_out + (size_t)q * n;
        memcpy(x, spins_in + (size_t)parent[s] * n, (size_t)n);
        E_out[q] = E[parent[s]];
    }
    for (int32_t sw = 0; sw < S; ++sw)
        for (int32_t q = 0; q < nsub; ++q)
            acc += sweep_replica(&g, spins_out + (size_t)q * n, &E_out[q], T, seed, sub[q], k, sw);
    if (nlm_now && nlm_block > 0) {
        const double qb = exp(-2.0 * beta_k);
        for (int32_t q = 0; q < nsub; ++q)
            orc_block_move(n, rp, col, w, spins_out + (size_t)q * n, &E_out[q], nlm_block, qb,
                           block_seed_vertex(seed, k, sub[q], n), block_accept_word(seed, k, sub[q]), NULL);
    } else if (nlm_now) {
        int32_t *order = (int32_t *)malloc((size_t)R * sizeof(int32_t));
        int32_t *where = (int32_t *)malloc((size_t)R * sizeof(int32_t));
        orc_nlm_order(R, seed, k, order);
        for (int32_t r = 0; r < R; ++r) where[r] = -1;
        for (int32_t q = 0; q < nsub; ++q) where[sub[q]] = q;
        for (int32_t m = 0; 2 * m + 1 < R; ++m) {
            int32_t a = order[2 * m], b = order[2 * m + 1];
            if (where[a] < 0 && where[b] < 0) continue;
            if (where[a] < 0 || where[b] < 0) { rc = -3; continue; }
            int8_t *xa = spins_out + (size_t)where[a] * n, *xb = spins_out + (size_t)where[b] * n;
            if (orc_houdayer_pair(n, rp, col, xa, xb, nlm_seed_word(seed, k, m), NULL) > 0) {
                E_out[where[a]] = (int32_t)orc_energy(n, rp, col, w, xa);
                E_out[where[b]] = (int32_t)orc_energy(n, rp, col, w, xb);
            }
        }
        free(order);
        free(where);
    }
    if (accepts_out) *accepts_out = acc;
    free(E); free(parent); free(T);
    free_view(&g);
    return rc;
}
