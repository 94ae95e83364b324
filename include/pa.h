/*
 * pa.h -- C ABI of libpa.so: Population Annealing Monte Carlo (PAMC) for
 * Max-Cut on one GB300 GPU (hand-written CUDA for sm_103a).
 *
 * Method (arXiv 2510.21105):
 *   Eq. 1   Max-Cut: maximise 1/2 sum_{i<j} w_ij (1 - x_i x_j), x in {-1,+1}^N.
 *   Sec. 2  Equivalently minimise the Ising energy with couplings -w_ij:
 *           E(x) = sum_{i<j} w_ij x_i x_j, and cut(x) = (W - E(x)) / 2 with
 *           W = sum_{i<j} w_ij.
 *   Sec. 3  The solver is PAMC (a population of replicas annealed in inverse
 *           temperature beta with Metropolis sweeps and Boltzmann
 *           resampling between temperatures), with adaptive control of
 *           stochasticity and periodic non-local moves, on one GPU. The
 *           paper defines these steps no further; the library implements the
 *           readings documented per entry point below, and every random
 *           decision is a counter-based Philox4x32-10 word keyed by the seed,
 *           so results are bit-identical run to run and independent of launch
 *           configuration.
 *
 * Conventions (all entry points):
 *   - Return 0 (PA_OK) on success or a negative PA_E* code. pa_strerror()
 *     names a code; pa_last_error() gives the detail of the last failure on a
 *     context. A failed call leaves previously returned results unchanged.
 *   - Host pointers are read or written synchronously and never retained:
 *     the caller owns every array it passes. Device memory is owned by the
 *     context and released by pa_destroy().
 *   - Vertices are numbered 0..n-1 (the paper numbers them 1..N).
 *   - The graph is CSR with every undirected edge stored in both rows:
 *     row_ptr[n+1] (uint32, row_ptr[0] = 0), col[row_ptr[n]] (uint16
 *     neighbour indices, so n <= 65536), w[row_ptr[n]] (int8 weights +1/-1,
 *     or NULL for all +1). The two copies of an edge must carry the same
 *     weight.
 *   - One context drives one GPU: the device current at pa_create().
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_OK 0
#define PA_EINVAL (-1)   /* invalid argument (graph, schedule, sizes, options) */
#define PA_ENOMEM (-2)   /* device or host allocation failed */
#define PA_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define PA_ETIMEOUT (-4) /* a served request did not finish within its
                            timeout (pa_request.timeout_ms). No kernel waits
                            on a flag, a peer or another kernel, so no
                            device-side wait returns it */
#define PA_EBUSY (-5)    /* the server is at its admission limit */
#define PA_ESTATE (-6)   /* call out of order (e.g. pa_best before any sweep) */

typedef struct pa_ctx pa_ctx;

/* Sweep kernel variants. */
#define PA_VARIANT_I8 0   /* int8 spins + int16/int8 local fields in shared memory */
#define PA_VARIANT_MSC 1  /* multi-spin coded: 32 replicas per 32-bit word */
#define PA_VARIANT_AUTO 2 /* chosen per graph and population: multi-spin coded
                             when the 32-replica words give every SM a word,
                             the CTA-pair kernel when they cover at least 40%
                             of the SMs, else the first of the packed byte
                             layout, int16 fields and multi-spin coding that
                             fits the graph in shared memory */
#define PA_VARIANT_MSC_PAIR 3 /* multi-spin coded, one thread-block cluster of two
                                 CTAs per 32-replica word (distributed shared
                                 memory); same results as PA_VARIANT_MSC */

typedef struct {
    int32_t variant;          /* PA_VARIANT_*; default PA_VARIANT_AUTO */
    int32_t field_bits;       /* I8 variant: shared-memory layout of a replica
                                 block: 16 = int8 spin + int16 field,
                                 8 = int8 spin + int8 field, 7 = one packed
                                 byte (spin bit + 7-bit field); 8 and 7 need
                                 max degree <= 127. 0 (default) = 7 when the
                                 degree allows, else 16. Results do not
                                 depend on the layout. */
    int32_t nlm_period;       /* non-local (Houdayer) move after the sweeps of
                                 step k when k > 0 and k % nlm_period == 0;
                                 0 = off (default) */
    int32_t adaptive;         /* 0 = schedule from betas[] (default);
                                 1 = ESS-adaptive temperature steps;
                                 2 = acceptance-rate-adaptive steps (same
                                 grid; the level moves one finer after a
                                 step that accepted less than acc_lo of its
                                 attempts, one coarser above acc_hi) */
    double rho;               /* adaptive: target ESS / R, in (0, 1] */
    int32_t adapt_J;          /* adaptive: finest level J (0..20) */
    double adapt_dbeta_max;   /* adaptive: coarsest step dbeta_max > 0 */
    double beta_max;          /* adaptive: final inverse temperature */
    int32_t replicas_per_cta; /* I8 variant: 4 or 8; 0 = auto */
    int32_t threads_per_cta;  /* 128..1024, multiple of 32; 0 = auto */
    void *stream;             /* cudaStream_t for every launch and copy;
                                 NULL = the legacy default stream */
    int32_t record_counts;    /* 1 = keep per-step copy counts (steps x R) */
    int32_t time_kernels;     /* 1 = time every sweep launch with CUDA events */
    int32_t nlm_kind;         /* non-local move (Sec. 3 names the moves only):
                                 0 = Houdayer cluster exchange between random
                                 replica pairs (default); 1 = block move: each
                                 replica flips the first nlm_block vertices of
                                 a breadth-first search from a random seed
                                 (rows scanned in CSR order) as one Metropolis
                                 move, accepted iff m <= 0 or u < A(m) with
                                 A(m) = min(2^32-1, floor(2^32 q^m)),
                                 q = exp(-2 beta_k) and m half the energy change */
    int32_t nlm_block;        /* block move size b, 1..1024 (default 32) */
    double acc_lo, acc_hi;    /* adaptive = 2: acceptance-rate band,
                                 0 <= acc_lo <= acc_hi <= 1 (0.05, 0.25) */
    int32_t reheat_after;     /* fixed schedules only: stagnation reheating.
                                 The schedule index advances one entry per
                                 step (staying at the last) unless this many
                                 consecutive steps found no lower energy at
                                 their sweep ends; then it steps back
                                 reheat_back entries (not below 0). Steps that
                                 do not advance resample with q = 1 (identity).
                                 0 = off (default) */
    int32_t reheat_back;      /* entries a reheat steps back (>= 1) */
    int32_t msc_no_split;     /* PA_VARIANT_MSC: 0 (default) = when the
                                 32-replica words are more than, and not a
                                 multiple of, the SMs, the first
                                 (words / SMs) * SMs words run in one-CTA
                                 blocks and the rest concurrently in CTA pairs
                                 on a second stream, so that every SM carries
                                 the same work; 1 = every word in one-CTA
                                 blocks, for callers whose other work (a
                                 batch, a loaded server) fills the SMs anyway.
                                 Results do not depend on it. */
} pa_anneal_opts;

typedef struct {
    int64_t attempts;         /* spin-flip attempts: n * R * sweeps * steps run */
    int64_t accepts;          /* accepted flips in all sweeps */
    int32_t steps_run;        /* temperature steps completed */
    int32_t n_colours;        /* colours of the greedy colouring */
    int32_t max_degree;
    int32_t kernel_launches;  /* library kernels launched by the anneal calls */
    int32_t sweep_launches;   /* of which sweep kernels */
    int32_t variant;          /* sweep variant actually used */
    double anneal_ms;         /* device time of the anneal calls (CUDA events) */
    double sweep_ms;          /* summed sweep-kernel time (time_kernels = 1) */
    double t_best_ms;         /* device time from the first step to the end of
                                 the step that recorded the final best */
    int64_t total_weight;     /* W = sum over undirected edges of w_ij */
    int64_t h2d_bytes;        /* host-to-device bytes copied by this context */
    int64_t d2h_bytes;        /* device-to-host bytes copied by this context */
} pa_stats_t;

/* Per-step records; each pointer may be NULL, arrays hold steps_run entries
 * (sweep_emin: steps_run * sweeps, counts: steps_run * R). */
typedef struct {
    double *beta;             /* beta_k used by the sweeps of step k */
    int32_t *emin;            /* minimum energy entering the resampling of step k */
    double *A;                /* FP64 weight sum A_k = sum_r exp(-dbeta (E_r - E_min)) */
    uint64_t *T;              /* integer weight total of the resampling */
    uint32_t *o;              /* systematic-resampling offset word */
    int64_t *accepts;         /* accepted flips in the sweeps of step k */
    double *lnZ;              /* free-energy estimate ln Z(beta_k) */
    int32_t *sweep_emin;      /* minimum energy over replicas after each sweep */
    int32_t *nlm_pairs;       /* non-local moves performed: pairs with D != {}
                                 (Houdayer) or accepted moves (block) */
    int64_t *nlm_flips;       /* spins flipped per replica by those moves */
    int32_t *jsel;            /* adaptive: chosen level j; reheating: the
                                 schedule index of step k; -1 otherwise */
    int32_t *counts;          /* copy counts n_r (record_counts = 1) */
    double *t_ms;             /* device time from the start of step 0 to the
                                 end of step k (global timer; includes any
                                 host gap between pa_anneal_run calls) */
} pa_step_arrays;

/* Fill *o with the defaults listed above. */
void pa_default_opts(pa_anneal_opts *o);

/* Create a context for one Max-Cut instance (Eq. 1; Ising form of Sec. 2).
 * Validates the CSR (n in 1..65536, row_ptr monotone, no self loops, no
 * duplicate neighbours, symmetric with equal weights, w in {+1,-1}), computes
 * the first-fit greedy colouring in vertex order (colour classes are the
 * parallel update sets of a sweep), renumbers vertices by colour, and copies
 * the graph to the current device. Errors: PA_EINVAL, PA_ENOMEM, PA_ECUDA;
 * *out is set only on success. */
int pa_create(pa_ctx **out, int32_t n, const uint32_t *row_ptr, const uint16_t *col,
              const int8_t *w);

/* Release the context and all its device memory (NULL is allowed). Waits
 * for the context's work to finish. */
void pa_destroy(pa_ctx *ctx);

/* Run a whole anneal: pa_anneal_begin() then pa_anneal_run(ctx, K), then
 * wait for completion. Sec. 3 (PAMC). Schedule: step k = 0..K-1 resamples
 * the population from beta_{k-1} to beta_k (beta_{-1} = 0, the initial i.i.d.
 * uniform population being exact at beta = 0), runs `sweeps` Metropolis
 * sweeps at beta_k (colour classes in order; a flip with energy change
 * dE = 2m is accepted iff m <= 0 or u < floor(2^32 exp(-2 beta_k m)), u a
 * uniform 32-bit integer whose top byte is byte slot%4 of word (slot/4)%4 of
 * Philox(vertex, slot/16, step, sweep) and whose low 24 bits, read only when
 * the top byte ties with the threshold's, are the top 24 bits of word slot%4
 * of Philox(vertex, slot/4, step, tag 4 | sweep)), records the best energy after
 * every sweep, and applies the non-local move when due.
 * betas: host array of K finite, non-negative, non-decreasing doubles
 * (ignored, may be NULL, when opts->adaptive = 1; K is then the maximum
 * number of steps). R: replicas, 1..65536. sweeps >= 0. opts: NULL =
 * defaults. Errors: PA_EINVAL, PA_ENOMEM, PA_ECUDA. */
int pa_anneal(pa_ctx *ctx, const double *betas, int32_t K, int32_t R, int32_t sweeps,
              uint64_t seed, const pa_anneal_opts *opts);

/* Allocate the population (R replicas, device resident), build the per-step
 * acceptance tables and resampling power tables on the host, and initialise
 * spins, local fields and energies on the device. No temperature step runs.
 * Arguments and errors as pa_anneal(). */
int pa_anneal_begin(pa_ctx *ctx, const double *betas, int32_t K, int32_t R, int32_t sweeps,
                    uint64_t seed, const pa_anneal_opts *opts);

/* Enqueue temperature steps [steps done, k_end) on the context's stream and
 * return without waiting for them (pa_sync waits). k_end is clamped to K.
 * In adaptive mode the steps after beta_max is reached are no-ops on the
 * device; so that they are not enqueued by the thousand, an adaptive run is
 * enqueued in chunks of 32 steps and the call waits (host side) until the
 * device is at most four chunks behind, reading whether the run has ended; it
 * then returns with the remaining steps counted as done. Not while the
 * stream is being captured (there every step is enqueued, without waits).
 * Errors: PA_ESTATE (no pa_anneal_begin), PA_EINVAL, PA_ECUDA. */
int pa_anneal_run(pa_ctx *ctx, int32_t k_end);

/* Wait for the context's stream; report a pending kernel error. */
int pa_sync(pa_ctx *ctx);

/* Best cut found so far (Sec. 3 reports one best cut and its configuration):
 * the lexicographic minimum of (energy, step, sweep, slot) over all sweep
 * ends. cut = (W - E*) / 2. config (may be NULL): host int8[n] of +1/-1 in
 * vertex order. step, sweep (may be NULL): where it was first recorded.
 * Waits for pending work. Errors: PA_ESTATE if no sweep has run. */
int pa_best(pa_ctx *ctx, int64_t *cut, int8_t *config, int32_t *step, int32_t *sweep);

/* As pa_best, also returning the best energy and the slot that held it. */
int pa_best_record(pa_ctx *ctx, int32_t *energy, int32_t *step, int32_t *sweep, int32_t *slot);

/* Copy the current population to the host: spins int8[R][n] (+1/-1, vertex
 * order; may be NULL) and energies int32[R] (may be NULL). Waits for pending
 * work. Errors: PA_ESTATE before pa_anneal_begin. */
int pa_get_state(pa_ctx *ctx, int8_t *spins, int32_t *energies);

/* Replace the population by host spins int8[R][n] (+1/-1, vertex order) and
 * mark `steps_done` steps as completed (resume / replay). Fields and energies
 * are recomputed on the device. Errors: PA_ESTATE, PA_EINVAL. */
int pa_set_state(pa_ctx *ctx, const int8_t *spins, int32_t steps_done);

/* Energies E = sum over edges w_ij x_i x_j and cuts (W - E)/2 (Eq. 1 and
 * the sign convention of Sec. 2) of R host configurations int8[R][n] (+1/-1,
 * vertex order), evaluated on the device with the kernel that initialises a
 * population. Independent of any anneal: a verifier for configurations read
 * back from files (e.g. the hexadecimal format of Sec. 3). energies int32[R]
 * and cuts int64[R] are caller buffers; either may be NULL. R = 0 is a no-op.
 * Allocates R*(3n + 4) bytes of device memory for the call. Errors: PA_EINVAL
 * (spin not +1/-1, R < 0), PA_ENOMEM, PA_ECUDA. */
int pa_energies(pa_ctx *ctx, const int8_t *spins, int32_t R, int32_t *energies, int64_t *cuts);

/* Checkpoint: write the anneal parameters, the population and the best
 * record to `path`; pa_load restores them into a context created for the
 * same graph (resume is bit-exact because all randomness is counter based).
 * Errors: PA_ESTATE, PA_EINVAL (unreadable file or different graph). */
int pa_save(pa_ctx *ctx, const char *path);
int pa_load(pa_ctx *ctx, const char *path);

/* Parameters of the current anneal (any pointer may be NULL); useful after
 * pa_load. Errors: PA_ESTATE before pa_anneal_begin. */
int pa_run_info(pa_ctx *ctx, int32_t *R, int32_t *K, int32_t *sweeps, int32_t *steps_done);

/* Totals and timings of the anneal (waits for pending work). */
int pa_stats(pa_ctx *ctx, pa_stats_t *out);

/* Per-step records (waits for pending work). */
int pa_step_stats(pa_ctx *ctx, pa_step_arrays *out);

/* ---------------------------------------------------------------------------
 * Batched anneals: many instances (each its own pa_ctx) advance through their
 * temperature steps together. Step k of every job is enqueued before step
 * k+1 of any, round-robin over n_streams streams, so instances of uneven size
 * overlap on the device; with use_graph the whole multi-stream sequence is
 * captured into one CUDA graph and launched once. Each job's results are
 * read afterwards from its context (pa_best, pa_stats, ...) and are
 * bit-identical to the same job run alone with pa_anneal (all randomness is
 * keyed by seed, slot, step, sweep and vertex, never by scheduling).
 */
typedef struct {
    pa_ctx *ctx;              /* from pa_create; owned by the caller */
    const double *betas;      /* host, K entries (NULL in adaptive mode) */
    int32_t K, R, sweeps;
    uint64_t seed;
    pa_anneal_opts opts;      /* per-job options; opts.stream is ignored */
} pa_job;

typedef struct {
    int32_t n_streams;        /* 1..64; 0 = min(n_jobs, 16) */
    int32_t use_graph;        /* 1 = capture into one CUDA graph, launch once */
    void *stream;             /* origin stream; NULL = legacy default stream */
} pa_batch_opts;

/* Run all jobs to completion. elapsed_ms (may be NULL) receives the device
 * time from the first step to the last (CUDA events on the origin stream;
 * graph instantiation excluded). Errors: PA_EINVAL, PA_ENOMEM, PA_ECUDA (the
 * failing job's pa_last_error gives the detail). */
int pa_batch_anneal(const pa_job *jobs, int32_t n_jobs, const pa_batch_opts *opts, double *elapsed_ms);

/* ---------------------------------------------------------------------------
 * Serving: a background thread admits anneal requests as device memory frees
 * up (FIFO; admitted when the estimated footprint fits under the HBM budget
 * and fewer than n_streams requests run, or when nothing else runs), keeps
 * their populations resident, and advances every admitted request, each on
 * its own stream, by steps_per_tick temperature steps per tick, so requests
 * that arrive while others run overlap with them on the device (continuous
 * batching). A request with opts.variant = PA_VARIANT_AUTO that is admitted
 * while other requests run takes the multi-spin-coded layout with every word
 * in one-CTA blocks (msc_no_split = 1: the cheapest attempt on a shared
 * device; max degree <= 127); admitted alone it keeps the automatic choice.
 * Each result is bit-identical to the same request run alone with pa_anneal.
 * Times are host milliseconds since pa_server_start.
 */
typedef struct pa_server pa_server;

typedef struct {
    int32_t n;                /* graph as in pa_create (host arrays, copied */
    const uint32_t *row_ptr;  /* by pa_server_submit) */
    const uint16_t *col;
    const int8_t *w;
    const double *betas;      /* host, K entries (copied) */
    int32_t K, R, sweeps;
    uint64_t seed;
    pa_anneal_opts opts;      /* opts.stream is ignored */
    double timeout_ms;        /* > 0: cancel the request with PA_ETIMEOUT if it
                                 has not completed this long after admission
                                 (its enqueued work drains first); 0 = none */
} pa_request;

typedef struct {
    int64_t cut;              /* best cut (W - E*) / 2 */
    int32_t energy, step, sweep, slot;
    int32_t status;           /* PA_OK or the error of the request */
    int64_t attempts;         /* spin-flip attempts performed */
    double submit_ms, start_ms, finish_ms;
} pa_response;

typedef struct {
    int64_t submitted, admitted, completed, queued, running;
    int64_t bytes_in_use;     /* estimated device bytes of admitted requests */
    int64_t attempts;         /* attempts of completed requests */
    double elapsed_ms;
} pa_server_stats_t;

/* Start the server on the current device. hbm_budget_bytes > 0; n_streams
 * = maximum concurrently running requests, 0..64 (0 = 16); steps_per_tick
 * >= 0 (0 = 8). */
int pa_server_start(pa_server **out, size_t hbm_budget_bytes, int32_t n_streams, int32_t steps_per_tick);
/* Queue a request (inputs are copied; returns at once). */
int pa_server_submit(pa_server *s, const pa_request *req, uint64_t *id);
/* state: 0 queued, 1 running, 2 done, negative = failed with that error. */
int pa_server_poll(pa_server *s, uint64_t id, int32_t *state);
/* Result of a finished request (config: host int8[n] or NULL). PA_EBUSY if
 * it has not finished. */
int pa_server_result(pa_server *s, uint64_t id, pa_response *out, int8_t *config);
/* Forget a finished request (its response and configuration); the server
 * already released its device memory and input copies when it finished.
 * PA_EBUSY if it has not finished, PA_EINVAL for an unknown id. */
int pa_server_release(pa_server *s, uint64_t id);
/* Testing hook for failure handling: while hold != 0 the tick thread enqueues
 * no further steps of request id, as if the host side of its job had stalled
 * (work already enqueued completes normally). A held request with a timeout
 * is cancelled with PA_ETIMEOUT; the others are not affected. */
int pa_server_hold(pa_server *s, uint64_t id, int32_t hold);
int pa_server_stats(pa_server *s, pa_server_stats_t *out);
/* Finish all submitted requests, then stop the thread and free everything. */
int pa_server_stop(pa_server *s);

/* Host-side copies of the tables the device uses for step k: the 32-bit
 * acceptance thresholds T[0..max_degree] and the 32 squarings q^(2^b) of
 * q = exp(-(beta_k - beta_{k-1})) used for the resampling weights. Either
 * pointer may be NULL. Errors: PA_ESTATE, PA_EINVAL. */
int pa_tables(pa_ctx *ctx, int32_t k, uint32_t *accept, double *qpow);

/* Colouring and renumbering chosen by pa_create: colour[n] per vertex,
 * position[n] of each vertex in the colour-sorted order (either may be
 * NULL). Returns the number of colours, or a negative error. */
int pa_colouring(pa_ctx *ctx, int32_t *colour, int32_t *position);

/* Device allocator hook (e.g. a framework's caching allocator). alloc
 * returns device memory of at least `bytes` bytes aligned to 256 bytes or
 * NULL; free releases it. Applies to allocations made after the call; NULL
 * functions restore cudaMalloc / cudaFree. Not thread safe against
 * concurrent allocations. */
typedef void *(*pa_alloc_fn)(size_t bytes, void *user);
typedef void (*pa_free_fn)(void *ptr, void *user);
void pa_set_allocator(pa_alloc_fn alloc, pa_free_fn free_fn, void *user);

/* ---------------------------------------------------------------------------
 * Resampling step without any device allocation.
 *
 * The paper has no counterpart to this entry point. It serves callers that
 * cannot call cudaMalloc: a host framework that owns the whole device-memory
 * budget through its own pool (a caching allocator that must see every byte,
 * so a library allocating on the side can push it out of memory), and
 * latency-critical loops where an allocator call may block, synchronise the
 * device or fail at a moment the caller cannot handle. It performs the same
 * reweighting and systematic resampling as one temperature step of
 * pa_anneal (weights exp(-(beta_k - beta_prev)(E_r - E_min)) as FP64
 * products of squarings, pairwise-tree weight sum, integer weights
 * floor(2^32 w_r), offset word from Philox(0, 0, k, tag 1) keyed by seed) and
 * returns bit-identical copy counts and parents.
 *
 *   energies  device int32[R]: energies of the population entering step k
 *   R         1..PA_NOALLOC_MAX_R (larger R returns PA_EINVAL)
 *   beta_prev, beta_k   finite, 0 <= beta_prev <= beta_k (else PA_EINVAL)
 *   seed, k   key and step index of the offset word
 *   parent    device int32[R]: new slot s receives old slot parent[s]
 *   counts    device int32[R] copy counts, or NULL
 *   out       host result (weight sum A, integer total T, E_min, offset o),
 *             or NULL; when given, the call copies it back and waits for the
 *             stream; with NULL the call only enqueues work and returns
 *   stream    cudaStream_t, NULL = legacy default stream
 *
 * Scratch lives in a fixed file-scope device array of about 0.6 MB that every
 * GPU loading the library holds until the process exits; no cudaMalloc,
 * cudaFree or allocating library routine is called. The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current, so make the first call on each device before any stream
 * capture. All calls share the array and it keeps the last call's contents;
 * every call writes each scratch word before reading it, so nothing needs
 * clearing between calls. Calls that overlap on the GPU (other streams, other
 * threads) race on it. Returns PA_OK, PA_EINVAL or PA_ECUDA.
 */
#define PA_NOALLOC_MAX_R 32768

typedef struct {
    double A;        /* FP64 weight sum */
    uint64_t T;      /* sum of integer weights */
    int32_t emin;    /* minimum energy */
    uint32_t o;      /* systematic-resampling offset word */
} pa_resample_result;

int pa_resample_noalloc(const int32_t *energies, int32_t R, double beta_prev, double beta_k,
                        uint64_t seed, int32_t k, int32_t *parent, int32_t *counts,
                        pa_resample_result *out, void *stream);

/* ---------------------------------------------------------------------------
 * Resampling of one population split over G ranks (replica sharding across
 * GPUs). Sec. 3 runs population annealing on one GPU; the reweighting and
 * systematic resampling here are those of pa_anneal (weights
 * q^(E - E_min) as FP64 products of squarings, pairwise tree sum A, integer
 * weights t = floor(2^32 w), copies F(P + t) - F(P) with
 * F(P) = floor((P R 2^32 + o T) / (T 2^32))), computed shard by shard so that
 * every output equals the single-population resampling bit for bit.
 *
 * Layout: R = 2^a replicas (R <= 65536) over G = 2^b ranks (G <= R, G <=
 * PA_SHARD_MAX_RANKS); rank g holds slots [g R/G, (g+1) R/G), one subtree of
 * the pairwise weight tree. One step on rank g (the caller does the three
 * collectives, e.g. with torch.distributed):
 *   pa_shard_min      -> E_min,g; all-reduce min -> E_min
 *   pa_shard_partials -> A_g, T_g (+ t and its prefix in scratch); all-gather
 *   pa_shard_plan     -> A, T, the new slots [new_lo, new_hi) this rank's
 *                        parents fill (contiguous: systematic resampling keeps
 *                        parent order) and the rows sent to / received from
 *                        every rank
 *   pa_shard_parents  -> local parent of each of those new slots
 *   pa_shard_gather   -> rows in new-slot order; all-to-all with the plan's
 *                        counts; rows arrive in new-slot order.
 * Device pointers: energies int32[n], scratch of pa_shard_scratch_bytes(n)
 * bytes (caller-owned, kept between pa_shard_partials and pa_shard_parents),
 * src int32[new_hi - new_lo] (may be empty: a rank whose parents fill no new
 * slot gathers nothing), counts int32[n] or NULL. stream: cudaStream_t or
 * NULL. pa_shard_plan and pa_resample_offset are host-only and need no GPU.
 * Errors: PA_EINVAL (sizes, layout, schedule), PA_ECUDA.
 */
#define PA_SHARD_MAX_RANKS 64
#define PA_SHARD_MAX_SLOTS 65536

typedef struct {
    double A;                 /* weight sum of the whole population (bitwise) */
    uint64_t T;               /* integer weight total of the whole population */
    uint64_t P_base;          /* integer weights of the ranks before this one */
    int32_t new_lo, new_hi;   /* new slots filled by this rank's parents */
    int32_t send[PA_SHARD_MAX_RANKS];   /* rows to rank h (new-slot order) */
    int32_t recv[PA_SHARD_MAX_RANKS];   /* rows from rank h (new-slot order) */
} pa_shard_step;

size_t pa_shard_scratch_bytes(int32_t n);
int pa_shard_min(const int32_t *energies, int32_t n, int32_t *scratch, int32_t *emin, void *stream);
int pa_shard_partials(const int32_t *energies, int32_t n, int32_t emin, double beta_prev, double beta_k,
                      void *scratch, double *A, uint64_t *T, void *stream);
int pa_shard_plan(int32_t G, int32_t g, int32_t R, const double *A_all, const uint64_t *T_all, uint32_t o,
                  pa_shard_step *out);
int pa_shard_parents(const void *scratch, int32_t n, int32_t R, uint32_t o, const pa_shard_step *step,
                     int32_t *src, int32_t *counts, void *stream);
int pa_shard_gather(const int8_t *spins, const int32_t *energies, int32_t ncols, const int32_t *src, int32_t nout,
                    int8_t *spins_out, int32_t *energies_out, void *stream);
/* Offset word o of the resampling of step k: word 0 of Philox(0, 0, k, tag 1)
 * keyed by the seed (host). */
uint32_t pa_resample_offset(uint64_t seed, int32_t k);

/* ---------------------------------------------------------------------------
 * Throughput probes of the current device (no counterpart in the paper; they
 * give the roofline denominators of the sweep, which is bound by integer
 * issue): register-only and shared-memory-only loops, four 256-thread CTAs per
 * SM, best of three launches timed with CUDA events on `stream` (NULL =
 * legacy default stream). Takes a few tens of milliseconds; allocates nothing.
 * Errors: PA_EINVAL (out NULL), PA_ECUDA.
 */
typedef struct {
    double int_ops_per_s;      /* 32-bit integer instructions per second, 1:1 mix
                                  of multiply-adds (IMAD) and three-input logic
                                  ops (LOP3), eight independent chains a thread */
    double philox_words_per_s; /* Philox4x32-10 output words per second */
    double smem_bytes_per_s;   /* shared-memory load bandwidth, 16-byte loads */
    int32_t sms;               /* multiprocessors of the device */
} pa_peaks;

int pa_probe_peaks(pa_peaks *out, void *stream);

/* Text of an error code, and the detail of the last error on ctx. */
const char *pa_strerror(int code);
const char *pa_last_error(const pa_ctx *ctx);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t pa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PA_H */
