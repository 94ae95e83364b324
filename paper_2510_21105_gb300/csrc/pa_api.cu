// pa_api.cu -- host side of libpa.so: the C ABI declared in include/pa.h.
//
// Graph preparation (validation, first-fit greedy colouring in vertex order,
// renumbering by colour), the per-step host tables (acceptance thresholds
// floor(2^32 exp(-beta_k 2m)) and the squarings of q_k = exp(-dbeta_k)), the
// device population, and the launch sequence of one temperature step:
//   resample (3 small kernels) -> sweep kernel (fused parent copy + S sweeps
//   + best tracking) -> non-local move when due.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pa.h"
#include "pa_internal.cuh"
#include "pa_moves.cuh"

namespace {

pa_alloc_fn g_alloc = nullptr;
pa_free_fn g_free = nullptr;
void *g_alloc_user = nullptr;

// Default device allocator: stream-ordered (cudaMallocAsync / cudaFreeAsync on
// the owning context's stream), so releasing a finished context never
// synchronises the device; the default pool keeps freed memory for reuse.
void *dev_alloc(size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    if (g_alloc) return g_alloc(bytes, g_alloc_user);
    static std::once_flag pool_once;
    std::call_once(pool_once, []() {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Frees are enqueued on the legacy default stream. Every caller has already
// synchronised the owning context's stream (pa_destroy, and pa_anneal_begin
// before it regrows a buffer), so no work still uses the memory; no stream
// handle is kept, since the stream an allocation was made on (for example a
// batch's temporary stream) may no longer exist when the buffer is freed.
void dev_free(void *p) {
    if (!p) return;
    if (g_free)
        g_free(p, g_alloc_user);
    else
        cudaFreeAsync(p, nullptr);
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        dev_free(p);
        p = nullptr;
        bytes = 0;
    }
    bool alloc(size_t b, cudaStream_t stream = nullptr) {
        if (p && bytes >= b) return true;
        release();
        p = dev_alloc(b, stream);
        if (!p) return false;
        bytes = b;
        return true;
    }
    template <class T>
    T *as() const {
        return reinterpret_cast<T *>(p);
    }
};

}  // namespace

struct RunState {
    bool begun = false;
    int32_t R = 0, Rpad = 0, K = 0, S = 0, nblk = 0, nch = 0, k_done = 0;
    int32_t nrec = 0;                    // replica blocks in all (one best record each)
    // Multi-spin coding with a word count that the SM count does not divide:
    // the first (words / SMs) * SMs words run in the one-CTA kernel and the
    // rest in the CTA-pair kernel on a second stream, concurrently, so every
    // SM carries the same share.
    bool split = false;
    // Adaptive runs end on the device (the controller reaches beta_max); the
    // host reads the active flag of a step behind the ones it enqueues, through
    // pinned slots, and stops enqueueing no-op steps (pa_anneal_run).
    int32_t *end_flag = nullptr;         // pinned [END_WINDOW]
    cudaEvent_t end_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    pa::SweepConfig sweep2{};
    int32_t nblk2 = 0, blk_base2 = 0;
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    uint64_t seed = 0;
    pa_anneal_opts opts{};
    std::vector<double> betas;           // per step (fixed schedule)
    std::vector<uint32_t> tables;        // [ntables][mmax+1]
    std::vector<double> qpow;            // [nq][32]
    std::vector<double> qblk;            // [ntables] exp(-2 beta) of each table row (block moves)
    int32_t ntables = 0, nq = 0;
    // device
    DevBuf spins[2], fields[2], E[2], parent;
    DevBuf partA, partT, tval, ploc;
    DevBuf d_tables, d_tidx, d_qpow, d_qblk;
    DevBuf rec_emin, rec_A, rec_T, rec_o, rec_acc, rec_sweep, rec_stamp, rec_counts;
    DevBuf rec_nlm_pairs, rec_nlm_flips, rec_jsel;
    DevBuf best_rec, best_cfg;
    DevBuf nlm_scratch;
    // adaptive
    DevBuf ad_state, ad_qsel, ad_active, ad_beta, ad_part;
    DevBuf d_betas;                      // reheating: the schedule on the device
    double ad_delta = 0.0;
    int32_t ad_nmax = 0;
    int cur = 0;
    pa::SweepConfig sweep{};
    int variant = PA_VARIANT_I8;
    // accounting
    int32_t launches = 0, sweep_launches = 0;
    double anneal_ms = 0.0, sweep_ms = 0.0;
    std::vector<cudaEvent_t> ev_pending;  // (start, end) pairs of anneal calls
    std::vector<cudaEvent_t> ev_sweep;    // (start, end) pairs of sweep launches
};

struct pa_ctx {
    int device = 0;
    int32_t n = 0, np = 0, m2 = 0, maxdeg = 0, ncol = 0;
    int64_t W = 0;
    bool weighted = false;
    uint64_t graph_hash = 0;
    std::vector<int32_t> colour, pos;   // per original vertex
    std::vector<uint32_t> vid;          // per position
    std::vector<int32_t> cls;           // [ncol+1]
    std::vector<uint32_t> rp_p;         // position-order CSR
    std::vector<uint16_t> col_p;
    std::vector<int8_t> w_p;
    DevBuf d_rp, d_col, d_w, d_vid, d_cls, d_pos, d_parity, d_prp, d_pcol, d_mrp, d_mcol;
    bool packed_ok = false, msc_rows = false;
    RunState run;
    std::string err;
    int64_t h2d = 0, d2h = 0;
    cudaStream_t stream() const { return reinterpret_cast<cudaStream_t>(run.opts.stream); }
    pa::GraphDev gdev() const {
        pa::GraphDev g;
        g.n = n;
        g.np = np;
        g.ncol = ncol;
        g.mmax = maxdeg;
        g.rp = d_rp.as<uint32_t>();
        g.col = d_col.as<uint16_t>();
        g.wt = weighted ? d_w.as<int8_t>() : nullptr;
        g.vid = d_vid.as<uint32_t>();
        g.cls = d_cls.as<int32_t>();
        g.parity = d_parity.as<uint32_t>();
        g.prp = d_prp.as<uint32_t>();
        g.pcol = d_pcol.as<uint2>();
        g.packed_ok = packed_ok ? 1 : 0;
        g.mrp = msc_rows ? d_mrp.as<uint32_t>() : nullptr;
        g.mcol = msc_rows ? d_mcol.as<uint2>() : nullptr;
        return g;
    }
};

namespace {

// cudaMemcpy / cudaMemcpyAsync with per-context byte accounting.
cudaError_t copy(pa_ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                 cudaStream_t st = nullptr, bool async = false) {
    if (kind == cudaMemcpyHostToDevice) c->h2d += (int64_t)bytes;
    if (kind == cudaMemcpyDeviceToHost) c->d2h += (int64_t)bytes;
    return async ? cudaMemcpyAsync(dst, src, bytes, kind, st) : cudaMemcpy(dst, src, bytes, kind);
}

int fail(pa_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(pa_ctx *c, cudaError_t e, const char *where) {
    return fail(c, PA_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PA_CUDA(ctx, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

uint64_t fnv1a(uint64_t h, const void *data, size_t bytes) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < bytes; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Acceptance thresholds of one inverse temperature.
void accept_row(double beta, int32_t mmax, uint32_t *row) {
    row[0] = 0xFFFFFFFFu;
    for (int32_t m = 1; m <= mmax; ++m) {
        const double p = std::exp(-(beta * (double)(2 * m)));
        const double v = std::floor(std::ldexp(p, 32));
        row[m] = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
    }
}

// Squarings s_0 = q, s_{b+1} = s_b * s_b of q.
void qpow_row(double q, double *row) {
    double s = q;
    for (int b = 0; b < 32; ++b) {
        row[b] = s;
        s = s * s;
    }
}

void free_run_events(RunState &r) {
    for (cudaEvent_t e : r.ev_pending) cudaEventDestroy(e);
    for (cudaEvent_t e : r.ev_sweep) cudaEventDestroy(e);
    r.ev_pending.clear();
    r.ev_sweep.clear();
    for (cudaEvent_t &e : r.end_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (r.end_flag) {
        cudaFreeHost(r.end_flag);
        r.end_flag = nullptr;
    }
}

// Fold finished event pairs into the timing totals (call after a sync).
void collect_events(RunState &r) {
    for (size_t i = 0; i + 1 < r.ev_pending.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.ev_pending[i], r.ev_pending[i + 1]) == cudaSuccess)
            r.anneal_ms += ms;
    }
    for (size_t i = 0; i + 1 < r.ev_sweep.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.ev_sweep[i], r.ev_sweep[i + 1]) == cudaSuccess)
            r.sweep_ms += ms;
    }
    cudaGetLastError();
    free_run_events(r);
}

int validate_opts(pa_ctx *c, const pa_anneal_opts &o) {
    if (o.variant < 0 || o.variant > 3) return fail(c, PA_EINVAL, "variant");
    if (o.field_bits != 16 && o.field_bits != 8 && o.field_bits != 7)
        return fail(c, PA_EINVAL, "field_bits must be 0, 16, 8 or 7");
    if (o.field_bits != 16 && c->maxdeg > 127)
        return fail(c, PA_EINVAL, "8- and 7-bit fields need max degree <= 127");
    if (o.field_bits == 7 && !c->packed_ok)
        return fail(c, PA_EINVAL, "the packed layout needs n <= 32720");
    const bool msc = o.variant == PA_VARIANT_MSC || o.variant == PA_VARIANT_MSC_PAIR;
    if (msc && c->maxdeg > 127)
        return fail(c, PA_EINVAL, "the multi-spin-coded variant needs max degree <= 127");
    if (msc && o.threads_per_cta > 256)
        return fail(c, PA_EINVAL, "the multi-spin-coded variant runs at most 256 threads per CTA");
    if (o.nlm_period < 0) return fail(c, PA_EINVAL, "nlm_period < 0");
    if (o.nlm_kind != 0 && o.nlm_kind != 1) return fail(c, PA_EINVAL, "nlm_kind must be 0 or 1");
    if (o.nlm_kind == 1 && (o.nlm_block < 1 || o.nlm_block > 1024))
        return fail(c, PA_EINVAL, "nlm_block must be 1..1024");
    if (o.replicas_per_cta != 0 && o.replicas_per_cta != 4 && o.replicas_per_cta != 8)
        return fail(c, PA_EINVAL, "replicas_per_cta must be 0, 4 or 8");
    if (o.threads_per_cta != 0 &&
        (o.threads_per_cta < 128 || o.threads_per_cta > 1024 || o.threads_per_cta % 32))
        return fail(c, PA_EINVAL, "threads_per_cta");
    if (o.adaptive < 0 || o.adaptive > 2) return fail(c, PA_EINVAL, "adaptive must be 0, 1 or 2");
    if (o.adaptive == 2 && !(o.acc_lo >= 0.0 && o.acc_lo <= o.acc_hi && o.acc_hi <= 1.0))
        return fail(c, PA_EINVAL, "acceptance band needs 0 <= acc_lo <= acc_hi <= 1");
    if (o.reheat_after < 0) return fail(c, PA_EINVAL, "reheat_after < 0");
    if (o.reheat_after > 0 && o.adaptive) return fail(c, PA_EINVAL, "reheating needs a fixed schedule");
    if (o.reheat_after > 0 && o.reheat_back < 1) return fail(c, PA_EINVAL, "reheat_back must be >= 1");
    if (o.msc_no_split != 0 && o.msc_no_split != 1) return fail(c, PA_EINVAL, "msc_no_split must be 0 or 1");
    if (o.adaptive) {
        if (!(o.rho > 0.0 && o.rho <= 1.0)) return fail(c, PA_EINVAL, "rho must be in (0, 1]");
        if (o.adapt_J < 0 || o.adapt_J > 20) return fail(c, PA_EINVAL, "adapt_J must be 0..20");
        if (!(o.adapt_dbeta_max > 0.0) || !std::isfinite(o.adapt_dbeta_max))
            return fail(c, PA_EINVAL, "adapt_dbeta_max");
        if (!(o.beta_max >= 0.0) || !std::isfinite(o.beta_max)) return fail(c, PA_EINVAL, "beta_max");
    }
    return PA_OK;
}

}  // namespace

extern "C" {

int32_t pa_version(void) { return 10000; }

const char *pa_strerror(int code) {
    switch (code) {
        case PA_OK: return "ok";
        case PA_EINVAL: return "invalid argument";
        case PA_ENOMEM: return "out of memory";
        case PA_ECUDA: return "CUDA error";
        case PA_ETIMEOUT: return "device wait timed out";
        case PA_EBUSY: return "server at admission limit";
        case PA_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

const char *pa_last_error(const pa_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

void pa_set_allocator(pa_alloc_fn alloc, pa_free_fn free_fn, void *user) {
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = user;
}

void pa_default_opts(pa_anneal_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->variant = PA_VARIANT_AUTO;
    o->field_bits = 0;
    o->rho = 0.5;
    o->adapt_J = 8;
    o->adapt_dbeta_max = 0.05;
    o->nlm_block = 32;
    o->acc_lo = 0.05;
    o->acc_hi = 0.25;
}

int pa_create(pa_ctx **out, int32_t n, const uint32_t *row_ptr, const uint16_t *col, const int8_t *w) {
    if (!out || !row_ptr || n < 1 || n > 65536) return PA_EINVAL;
    if (row_ptr[0] != 0) return PA_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return PA_EINVAL;
    const uint32_t m2 = row_ptr[n];
    if (m2 > 0 && !col) return PA_EINVAL;
    if (m2 > 0x7FFFFFFFu) return PA_EINVAL;
    // Self loops, range, duplicates, weights.
    std::vector<int32_t> mark(n, -1);
    int32_t maxdeg = 0;
    for (int32_t i = 0; i < n; ++i) {
        maxdeg = std::max<int32_t>(maxdeg, (int32_t)(row_ptr[i + 1] - row_ptr[i]));
        for (uint32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t j = col[e];
            if (j >= n || j == i || mark[j] == i) return PA_EINVAL;
            mark[j] = i;
            if (w && w[e] != 1 && w[e] != -1) return PA_EINVAL;
        }
    }
    if (maxdeg > 32767) return PA_EINVAL;
    // Symmetry with equal weights: sort (min, max, w) of every stored entry.
    {
        std::vector<uint64_t> keys;
        keys.reserve(m2);
        for (int32_t i = 0; i < n; ++i)
            for (uint32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const uint64_t a = (uint64_t)std::min<int32_t>(i, col[e]);
                const uint64_t b = (uint64_t)std::max<int32_t>(i, col[e]);
                const uint64_t s = (w && w[e] < 0) ? 1u : 0u;
                keys.push_back((a << 33) | (b << 1) | s);
            }
        std::sort(keys.begin(), keys.end());
        if (keys.size() % 2) return PA_EINVAL;
        for (size_t t = 0; t < keys.size(); t += 2)
            if (keys[t] != keys[t + 1] || (t + 2 < keys.size() && (keys[t + 2] >> 1) == (keys[t] >> 1)))
                return PA_EINVAL;
    }
    pa_ctx *c = new (std::nothrow) pa_ctx();
    if (!c) return PA_ENOMEM;
    cudaGetDevice(&c->device);
    c->n = n;
    c->np = (n + 15) & ~15;
    c->m2 = (int32_t)m2;
    c->maxdeg = maxdeg;
    c->weighted = false;
    if (w)
        for (uint32_t e = 0; e < m2; ++e)
            if (w[e] < 0) { c->weighted = true; break; }
    // W = sum over undirected edges.
    int64_t W2 = 0;
    for (uint32_t e = 0; e < m2; ++e) W2 += w ? w[e] : 1;
    c->W = W2 / 2;
    // First-fit greedy colouring in vertex order.
    c->colour.assign(n, 0);
    std::vector<int32_t> seen(n + 2, -1);
    int32_t ncol = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (uint32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] < i) seen[c->colour[col[e]]] = i;
        int32_t k = 0;
        while (seen[k] == i) ++k;
        c->colour[i] = k;
        ncol = std::max(ncol, k + 1);
    }
    c->ncol = ncol;
    // Renumber: positions sorted by (colour, degree descending, vertex). A colour
    // class is an independent set and every random number is keyed by the vertex,
    // so the order inside a class does not change any result; sorting by degree
    // gives the 32 lanes of a warp neighbour loops of nearly equal length.
    c->cls.assign(ncol + 1, 0);
    for (int32_t i = 0; i < n; ++i) c->cls[c->colour[i] + 1]++;
    for (int32_t k = 0; k < ncol; ++k) c->cls[k + 1] += c->cls[k];
    c->pos.assign(n, 0);
    c->vid.assign(n, 0);
    {
        std::vector<int32_t> fill(c->cls.begin(), c->cls.end() - 1);
        for (int32_t i = 0; i < n; ++i) c->vid[fill[c->colour[i]]++] = (uint32_t)i;
        for (int32_t k = 0; k < ncol; ++k)
            std::stable_sort(c->vid.begin() + c->cls[k], c->vid.begin() + c->cls[k + 1], [&](uint32_t a, uint32_t b) {
                return row_ptr[a + 1] - row_ptr[a] > row_ptr[b + 1] - row_ptr[b];
            });
        for (int32_t p = 0; p < n; ++p) c->pos[c->vid[p]] = p;
    }
    c->rp_p.assign(n + 1, 0);
    c->col_p.resize(m2);
    c->w_p.resize(m2);
    for (int32_t p = 0; p < n; ++p) {
        const int32_t i = (int32_t)c->vid[p];
        c->rp_p[p + 1] = c->rp_p[p] + (row_ptr[i + 1] - row_ptr[i]);
        uint32_t o = c->rp_p[p];
        for (uint32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e, ++o) {
            c->col_p[o] = (uint16_t)c->pos[col[e]];
            c->w_p[o] = w ? w[e] : 1;
        }
    }
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, &n, sizeof(n));
    h = fnv1a(h, row_ptr, sizeof(uint32_t) * (n + 1));
    if (m2) h = fnv1a(h, col, sizeof(uint16_t) * m2);
    if (w && m2) h = fnv1a(h, w, m2);
    c->graph_hash = h;
    // Upload.
    if (!c->d_rp.alloc(sizeof(uint32_t) * (n + 1)) || !c->d_col.alloc(sizeof(uint16_t) * (m2 + 8)) ||
        !c->d_w.alloc(m2 + 16) || !c->d_vid.alloc(sizeof(uint32_t) * n) ||
        !c->d_cls.alloc(sizeof(int32_t) * (ncol + 1)) || !c->d_pos.alloc(sizeof(int32_t) * n) ||
        !c->d_parity.alloc(sizeof(uint32_t) * ((c->np + 31) / 32))) {
        delete c;
        return PA_ENOMEM;
    }
    cudaError_t e1 = copy(c, c->d_rp.p, c->rp_p.data(), sizeof(uint32_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess && m2)
        e1 = copy(c, c->d_col.p, c->col_p.data(), sizeof(uint16_t) * m2, cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess && m2)
        e1 = copy(c, c->d_w.p, c->w_p.data(), m2, cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess)
        e1 = copy(c, c->d_vid.p, c->vid.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess)
        e1 = copy(c, c->d_cls.p, c->cls.data(), sizeof(int32_t) * (ncol + 1), cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess)
        e1 = copy(c, c->d_pos.p, c->pos.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
    c->packed_ok = c->np + 32 <= 32768;
    if (e1 == cudaSuccess && c->packed_ok) {
        std::vector<uint32_t> prp(n + 1, 0u);
        for (int32_t p = 0; p < n; ++p) prp[p + 1] = prp[p] + (c->rp_p[p + 1] - c->rp_p[p] + 3) / 4;
        std::vector<uint16_t> pcol((size_t)prp[n] * 4 + 4);
        for (int32_t p = 0; p < n; ++p) {
            size_t o = (size_t)prp[p] * 4;
            for (uint32_t e = c->rp_p[p]; e < c->rp_p[p + 1]; ++e, ++o)
                pcol[o] = (uint16_t)(c->col_p[e] | (c->w_p[e] < 0 ? 0x8000u : 0u));
            for (; o < (size_t)prp[p + 1] * 4; ++o) pcol[o] = (uint16_t)(c->np + (p & 31));
        }
        if (!c->d_prp.alloc(4 * (size_t)(n + 1)) || !c->d_pcol.alloc(2 * pcol.size())) {
            delete c;
            return PA_ENOMEM;
        }
        e1 = copy(c, c->d_prp.p, prp.data(), 4 * (size_t)(n + 1), cudaMemcpyHostToDevice);
        if (e1 == cudaSuccess) e1 = copy(c, c->d_pcol.p, pcol.data(), 2 * pcol.size(), cudaMemcpyHostToDevice);
    }
    c->msc_rows = c->np <= 16384 && c->maxdeg <= 127;
    if (e1 == cudaSuccess && c->msc_rows) {
        std::vector<uint32_t> mrp(n + 1, 0u);
        uint32_t units = 0;
        for (int32_t p = 0; p < n; ++p) {
            const uint32_t d = c->rp_p[p + 1] - c->rp_p[p];
            mrp[p] = units << 8 | d;
            units += (d + 3) / 4;
        }
        mrp[n] = units << 8;
        std::vector<uint16_t> mcol((size_t)units * 4 + 4);
        for (int32_t p = 0; p < n; ++p) {
            size_t o = (size_t)(mrp[p] >> 8) * 4;
            for (uint32_t e = c->rp_p[p]; e < c->rp_p[p + 1]; ++e, ++o)
                mcol[o] = (uint16_t)(4u * c->col_p[e] | (c->w_p[e] < 0 ? 1u : 0u));
            for (; o < (size_t)(mrp[p + 1] >> 8) * 4; ++o) mcol[o] = (uint16_t)(4u * (uint32_t)p);
        }
        if (!c->d_mrp.alloc(4 * (size_t)(n + 1)) || !c->d_mcol.alloc(2 * mcol.size())) {
            delete c;
            return PA_ENOMEM;
        }
        e1 = copy(c, c->d_mrp.p, mrp.data(), 4 * (size_t)(n + 1), cudaMemcpyHostToDevice);
        if (e1 == cudaSuccess) e1 = copy(c, c->d_mcol.p, mcol.data(), 2 * mcol.size(), cudaMemcpyHostToDevice);
    }
    if (e1 == cudaSuccess) {
        std::vector<uint32_t> par((c->np + 31) / 32, 0u);
        for (int32_t p = 0; p < n; ++p)
            if ((c->rp_p[p + 1] - c->rp_p[p]) & 1u) par[p >> 5] |= 1u << (p & 31);
        e1 = copy(c, c->d_parity.p, par.data(), sizeof(uint32_t) * par.size(), cudaMemcpyHostToDevice);
    }
    if (e1 != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return PA_ECUDA;
    }
    *out = c;
    return PA_OK;
}

void pa_destroy(pa_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream());
    free_run_events(ctx->run);
    RunState &r = ctx->run;
    if (r.st2) {
        cudaStreamSynchronize(r.st2);
        cudaStreamDestroy(r.st2);
    }
    if (r.ev_fork) cudaEventDestroy(r.ev_fork);
    if (r.ev_join) cudaEventDestroy(r.ev_join);
    cudaGetLastError();
    delete ctx;   // buffers return to the memory pool
}

int pa_anneal_begin(pa_ctx *c, const double *betas, int32_t K, int32_t R, int32_t sweeps,
                    uint64_t seed, const pa_anneal_opts *opts) {
    if (!c) return PA_EINVAL;
    pa_anneal_opts o;
    pa_default_opts(&o);
    if (opts) o = *opts;
    // Every layout keeps a replica block in shared memory, so the graph size
    // decides which layouts exist: multi-spin coding needs 4 bytes per vertex
    // (n up to about 57,000 on GB300), the packed byte 4 bytes per vertex and
    // n <= 32720, the int16 layout 12 bytes per vertex (n up to about 19,000).
    int dev = 0, sms = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (sms <= 0) sms = 152;
    if (smem_max <= 0) smem_max = 227 * 1024;
    const pa::GraphDev gd = c->gdev();
    auto fits = [&](int fb, int G, int th) { return pa::sweep_smem_bytes(gd, G, fb, th) <= (size_t)smem_max; };
    const bool msc_fits = c->maxdeg <= 127 && fits(1, 8, 256);
    const bool packed_fits = c->maxdeg <= 127 && c->packed_ok && fits(7, 1, o.threads_per_cta ? o.threads_per_cta : 128);
    const bool int16_fits = fits(16, o.replicas_per_cta == 8 ? 2 : 1, 512);
    if (o.variant == PA_VARIANT_AUTO) {
        // Multi-spin coding is fastest once its 32-replica words give every SM
        // at least one block (the words past the largest SM multiple run in the
        // CTA-pair kernel, see below). With fewer words, down to about 40% of
        // the SM count, the CTA-pair kernel (two CTAs per word) still beats the
        // 4-replica packed layout; below that the packed layout's smaller
        // blocks win. Measured (G attempts/s, packed / MSC / MSC pair):
        // G63-shaped R = 2048: 251 / 196 / 255; R = 4096: 357 / 388 / 413;
        // R = 8192: 362 / 558 / 533; torus 100x100 R = 2048: 281 / 265 / 445.
        const bool msc_ok = msc_fits && o.field_bits == 0 && (o.threads_per_cta == 0 || o.threads_per_cta <= 256);
        const int32_t words = (R + 31) / 32;
        if (msc_ok && words >= sms)
            o.variant = PA_VARIANT_MSC;
        else if (msc_ok && 5 * words >= 2 * sms)
            o.variant = PA_VARIANT_MSC_PAIR;
        else if ((o.field_bits == 0 || o.field_bits == 7) && packed_fits)
            o.variant = PA_VARIANT_I8;
        else if (o.field_bits == 0 && !int16_fits && msc_ok)
            o.variant = PA_VARIANT_MSC;   // the only layout that fits the graph
        else
            o.variant = PA_VARIANT_I8;
    }
    if (o.field_bits == 0) o.field_bits = (c->maxdeg <= 127 && c->packed_ok) ? 7 : 16;
    {
        const bool msc = o.variant == PA_VARIANT_MSC || o.variant == PA_VARIANT_MSC_PAIR;
        const int fb = msc ? 1 : o.field_bits;
        const int G = msc ? 8 : (o.replicas_per_cta == 8 ? 2 : 1);
        const int th = o.threads_per_cta ? o.threads_per_cta : (msc ? 256 : (o.field_bits == 7 ? 128 : 512));
        const size_t need = pa::sweep_smem_bytes(gd, G, fb, th);
        if (need > (size_t)smem_max)
            return fail(c, PA_EINVAL, "graph too large for this layout: a sweep block needs " + std::to_string(need) +
                                          " bytes of shared memory, the device allows " + std::to_string(smem_max));
    }
    if (K < 0 || R < 1 || R > 65536 || sweeps < 0 || sweeps >= (1 << 28))
        return fail(c, PA_EINVAL, "K, R (1..65536) or sweeps out of range");
    if (int rc = validate_opts(c, o)) return rc;
    if (o.nlm_period > 0 && o.nlm_kind == 0 && pa::nlm_smem_bytes(c->np) > 200 * 1024)
        return fail(c, PA_EINVAL, "Houdayer moves need " + std::to_string(pa::nlm_smem_bytes(c->np)) +
                                      " bytes of shared memory per replica pair, more than 200 KB");
    if (!o.adaptive) {
        if (K > 0 && !betas) return fail(c, PA_EINVAL, "betas is NULL");
        double prev = 0.0;
        for (int32_t k = 0; k < K; ++k) {
            if (!std::isfinite(betas[k]) || betas[k] < prev)
                return fail(c, PA_EINVAL, "betas must be finite, >= 0 and non-decreasing");
            prev = betas[k];
        }
    }
    RunState &r = c->run;
    cudaStreamSynchronize(c->stream());
    collect_events(r);
    r.begun = false;
    r.opts = o;
    r.R = R;
    r.K = K;
    r.S = sweeps;
    r.seed = seed;
    r.k_done = 0;
    r.launches = r.sweep_launches = 0;
    r.anneal_ms = r.sweep_ms = 0.0;
    r.variant = o.variant == PA_VARIANT_AUTO ? PA_VARIANT_I8 : o.variant;
    // Sweep kernel shape.
    const bool msc = o.variant == PA_VARIANT_MSC || o.variant == PA_VARIANT_MSC_PAIR;
    int G = o.replicas_per_cta == 8 ? 2 : 1;
    int threads = o.threads_per_cta ? o.threads_per_cta : (msc ? 256 : (o.field_bits == 7 ? 128 : 512));
    pa::GraphDev g = c->gdev();
    const int fcode = o.variant == PA_VARIANT_MSC_PAIR ? 2 : (msc ? 1 : o.field_bits);
    cudaError_t ce = pa::sweep_configure(g, R, G, fcode, threads, c->weighted, &r.sweep);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "sweep_configure");
    G = r.sweep.G;
    r.Rpad = ((R + 4 * G - 1) / (4 * G)) * 4 * G;
    r.nblk = r.Rpad / (4 * G);
    r.nrec = r.nblk;
    r.split = false;
    if (o.variant == PA_VARIANT_MSC && !o.msc_no_split) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int32_t words = r.nblk, wm = sms > 0 ? (words / sms) * sms : 0;
        if (wm > 0 && wm < words) {
            ce = pa::sweep_configure(g, R - 32 * wm, 8, 2, 256, c->weighted, &r.sweep2);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "sweep_configure (tail)");
            ce = pa::sweep_configure(g, 32 * wm, 8, 1, threads, c->weighted, &r.sweep);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "sweep_configure (head)");
            if (!r.st2 && cudaStreamCreateWithFlags(&r.st2, cudaStreamNonBlocking) != cudaSuccess)
                return fail(c, PA_ECUDA, "stream create");
            if (!r.ev_fork && cudaEventCreateWithFlags(&r.ev_fork, cudaEventDisableTiming) != cudaSuccess)
                return fail(c, PA_ECUDA, "event create");
            if (!r.ev_join && cudaEventCreateWithFlags(&r.ev_join, cudaEventDisableTiming) != cudaSuccess)
                return fail(c, PA_ECUDA, "event create");
            r.split = true;
            r.nblk = wm;
            r.nblk2 = words - wm;
            r.blk_base2 = wm;
        }
    }
    r.nch = (R + pa::RS_CHUNK - 1) / pa::RS_CHUNK;
    const int32_t mmax = c->maxdeg;
    // Host tables.
    if (!o.adaptive) {
        r.betas.assign(betas, betas + K);
        r.ntables = std::max(K, 1);
        r.tables.assign((size_t)r.ntables * (mmax + 1), 0u);
        // Reheating adds row K: q = 1 for steps that do not advance the schedule.
        r.nq = std::max(K, 1) + (o.reheat_after > 0 ? 1 : 0);
        r.qpow.assign((size_t)r.nq * 32, 0.0);
        double prev = 0.0;
        for (int32_t k = 0; k < K; ++k) {
            accept_row(betas[k], mmax, &r.tables[(size_t)k * (mmax + 1)]);
            qpow_row(std::exp(-(betas[k] - prev)), &r.qpow[(size_t)k * 32]);
            prev = betas[k];
        }
        if (o.reheat_after > 0) qpow_row(1.0, &r.qpow[(size_t)(r.nq - 1) * 32]);
    } else {
        r.betas.clear();
        r.ad_delta = std::ldexp(o.adapt_dbeta_max, -o.adapt_J);
        r.ad_nmax = (int32_t)std::floor(o.beta_max / r.ad_delta + 0.5);
        if ((double)(r.ad_nmax + 1) * (mmax + 1) * 4.0 > 2.0e9)
            return fail(c, PA_EINVAL, "adaptive grid too fine (acceptance tables exceed 2 GB)");
        r.ntables = r.ad_nmax + 1;
        r.tables.assign((size_t)r.ntables * (mmax + 1), 0u);
        for (int32_t n = 0; n <= r.ad_nmax; ++n)
            accept_row((double)n * r.ad_delta, mmax, &r.tables[(size_t)n * (mmax + 1)]);
        r.nq = (1 << o.adapt_J);   // row dn-1 holds the squarings of exp(-dn delta)
        r.qpow.assign((size_t)r.nq * 32, 0.0);
        for (int32_t dn = 1; dn <= r.nq; ++dn)
            qpow_row(std::exp(-((double)dn * r.ad_delta)), &r.qpow[(size_t)(dn - 1) * 32]);
    }
    // Block moves: q = exp(-2 beta) of every table row (beta_k, or n delta when adaptive).
    r.qblk.clear();
    if (o.nlm_period > 0 && o.nlm_kind == 1) {
        r.qblk.assign((size_t)r.ntables, 1.0);
        for (int32_t t = 0; t < r.ntables; ++t) {
            const double beta = o.adaptive ? (double)t * r.ad_delta : (t < K ? betas[t] : 0.0);
            r.qblk[t] = std::exp(-2.0 * beta);
        }
    }
    // Device buffers (stream-ordered on the context's stream).
    cudaStream_t ST = c->stream();
    const size_t npR = (size_t)c->np * r.Rpad;
    const int32_t Kc = std::max(K, 1);
    const int32_t Sc = std::max(sweeps, 1);
    const size_t nrs = (size_t)r.nch * pa::RS_CHUNK;
    bool ok = r.spins[0].alloc(npR, ST) && r.spins[1].alloc(npR, ST) && r.fields[0].alloc(2 * npR, ST) &&
              r.fields[1].alloc(2 * npR, ST) && r.E[0].alloc(4 * (size_t)r.Rpad, ST) &&
              r.E[1].alloc(4 * (size_t)r.Rpad, ST) && r.parent.alloc(4 * (size_t)r.Rpad, ST) &&
              r.partA.alloc(8 * (size_t)r.nch, ST) && r.partT.alloc(8 * (size_t)r.nch, ST) &&
              r.tval.alloc(8 * nrs, ST) && r.ploc.alloc(8 * nrs, ST) &&
              r.d_tables.alloc(4 * r.tables.size(), ST) && r.d_tidx.alloc(4 * (size_t)Kc, ST) &&
              r.d_qpow.alloc(8 * r.qpow.size(), ST) && r.rec_emin.alloc(4 * (size_t)Kc, ST) &&
              r.rec_A.alloc(8 * (size_t)Kc, ST) && r.rec_T.alloc(8 * (size_t)Kc, ST) &&
              r.rec_o.alloc(4 * (size_t)Kc, ST) && r.rec_acc.alloc(8 * (size_t)Kc, ST) &&
              r.rec_sweep.alloc(4 * (size_t)Kc * Sc, ST) && r.rec_stamp.alloc(8 * (size_t)(Kc + 1), ST) &&
              r.rec_nlm_pairs.alloc(4 * (size_t)Kc, ST) && r.rec_nlm_flips.alloc(8 * (size_t)Kc, ST) &&
              r.rec_jsel.alloc(4 * (size_t)Kc, ST) && r.best_rec.alloc(16 * (size_t)r.nrec, ST) &&
              r.best_cfg.alloc((size_t)r.nrec * c->np, ST);
    if (ok && o.record_counts) ok = r.rec_counts.alloc(4 * (size_t)Kc * R, ST);
    if (ok && o.adaptive)
        ok = r.ad_state.alloc(16, ST) && r.ad_qsel.alloc(4 * (size_t)Kc, ST) && r.ad_active.alloc(4 * (size_t)Kc, ST) &&
             r.ad_beta.alloc(8 * (size_t)Kc, ST) && r.ad_part.alloc(16 * (size_t)(o.adapt_J + 1) * r.nch, ST);
    if (ok && o.reheat_after > 0)
        ok = r.ad_state.alloc(16, ST) && r.ad_qsel.alloc(4 * (size_t)Kc, ST) && r.ad_beta.alloc(8 * (size_t)Kc, ST) &&
             r.d_betas.alloc(8 * (size_t)Kc, ST);
    if (ok && o.nlm_period > 0) ok = r.nlm_scratch.alloc(pa::nlm_scratch_bytes(R), ST);
    if (ok && !r.qblk.empty()) ok = r.d_qblk.alloc(8 * r.qblk.size(), ST);
    if (!ok) return fail(c, PA_ENOMEM, "device allocation failed");
    cudaStream_t st = c->stream();
    PA_CUDA(c, copy(c, r.d_tables.p, r.tables.data(), 4 * r.tables.size(), cudaMemcpyHostToDevice, st, true));
    PA_CUDA(c, copy(c, r.d_qpow.p, r.qpow.data(), 8 * r.qpow.size(), cudaMemcpyHostToDevice, st, true));
    if (!r.qblk.empty())
        PA_CUDA(c, copy(c, r.d_qblk.p, r.qblk.data(), 8 * r.qblk.size(), cudaMemcpyHostToDevice, st, true));
    {
        std::vector<int32_t> tidx(Kc);
        for (int32_t k = 0; k < Kc; ++k) tidx[k] = o.adaptive ? 0 : k;
        PA_CUDA(c, copy(c, r.d_tidx.p, tidx.data(), 4 * (size_t)Kc, cudaMemcpyHostToDevice, st, true));
        std::vector<int32_t> ident(r.Rpad);
        for (int32_t s = 0; s < r.Rpad; ++s) ident[s] = s;
        PA_CUDA(c, copy(c, r.parent.p, ident.data(), 4 * (size_t)r.Rpad, cudaMemcpyHostToDevice, st, true));
        std::vector<int4> br(r.nrec, make_int4(0x7FFFFFFF, -1, -1, -1));
        PA_CUDA(c, copy(c, r.best_rec.p, br.data(), 16 * (size_t)r.nrec, cudaMemcpyHostToDevice, st, true));
        // Pageable sources: wait before the vectors go out of scope.
        PA_CUDA(c, cudaStreamSynchronize(st));
    }
    PA_CUDA(c, cudaMemsetAsync(r.rec_emin.p, 0x7F, 4 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_sweep.p, 0x7F, 4 * (size_t)Kc * Sc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_acc.p, 0, 8 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_A.p, 0, 8 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_T.p, 0, 8 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_o.p, 0, 4 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_stamp.p, 0, 8 * (size_t)(Kc + 1), st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_nlm_pairs.p, 0, 4 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_nlm_flips.p, 0, 8 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.rec_jsel.p, 0xFF, 4 * (size_t)Kc, st));
    PA_CUDA(c, cudaMemsetAsync(r.best_cfg.p, 0, (size_t)r.nrec * c->np, st));
    if (o.record_counts) PA_CUDA(c, cudaMemsetAsync(r.rec_counts.p, 0, 4 * (size_t)Kc * R, st));
    if (o.reheat_after > 0) {
        PA_CUDA(c, cudaMemsetAsync(r.ad_state.p, 0, 16, st));
        PA_CUDA(c, cudaMemsetAsync(r.ad_qsel.p, 0, 4 * (size_t)Kc, st));
        PA_CUDA(c, cudaMemsetAsync(r.ad_beta.p, 0, 8 * (size_t)Kc, st));
        if (K > 0) PA_CUDA(c, copy(c, r.d_betas.p, r.betas.data(), 8 * (size_t)K, cudaMemcpyHostToDevice, st, true));
    }
    if (o.adaptive) {
        PA_CUDA(c, cudaMemsetAsync(r.ad_state.p, 0, 16, st));
        PA_CUDA(c, cudaMemsetAsync(r.ad_active.p, 0, 4 * (size_t)Kc, st));
        PA_CUDA(c, cudaMemsetAsync(r.ad_qsel.p, 0, 4 * (size_t)Kc, st));
        PA_CUDA(c, cudaMemsetAsync(r.ad_beta.p, 0, 8 * (size_t)Kc, st));
    }
    // Initial population at beta = 0, fields and energies.
    r.cur = 0;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    PA_CUDA(c, cudaMemsetAsync(r.spins[0].p, 0, npR, st));
    PA_CUDA(c, pa::launch_init(g, r.spins[0].as<int8_t>(), r.Rpad, k0, k1, st));
    PA_CUDA(c, pa::launch_fields(g, r.spins[0].as<int8_t>(), r.fields[0].as<int16_t>(), r.E[0].as<int32_t>(),
                                 r.Rpad, st));
    r.launches += 2;
    r.begun = true;
    return PA_OK;
}

}  // extern "C"

namespace {
// Enqueue temperature step k of the context's anneal on stream st.
int enqueue_step(pa_ctx *c, int32_t k, cudaStream_t st, bool time_sweep) {
    RunState &r = c->run;
    pa::GraphDev g = c->gdev();
    const uint32_t k0 = (uint32_t)r.seed, k1 = (uint32_t)(r.seed >> 32);
    const pa_anneal_opts &o = r.opts;
    const int cur = r.cur, nxt = 1 - r.cur;
    pa::ResampleArgs ra{};
    ra.E = r.E[cur].as<int32_t>();
    ra.R = r.R;
    ra.nch = r.nch;
    ra.k = k;
    ra.key0 = k0;
    ra.key1 = k1;
    ra.qpow = r.d_qpow.as<double>();
    ra.qsel = (o.adaptive || o.reheat_after > 0) ? r.ad_qsel.as<int32_t>() : nullptr;
    if (o.reheat_after > 0) {
        pa::ReheatArgs ha{};
        ha.sweep_emin = r.rec_sweep.as<int32_t>();
        ha.betas = r.d_betas.as<double>();
        ha.k = k;
        ha.K = r.K;
        ha.S = r.S;
        ha.after = o.reheat_after;
        ha.back = o.reheat_back;
        ha.state = r.ad_state.as<int32_t>();
        ha.tidx = r.d_tidx.as<int32_t>();
        ha.qsel = r.ad_qsel.as<int32_t>();
        ha.isel = r.rec_jsel.as<int32_t>();
        ha.beta = r.ad_beta.as<double>();
        PA_CUDA(c, pa::launch_reheat(ha, st));
        r.launches += 1;
    }
    ra.active = nullptr;   // the minimum runs before the adaptive decision
    ra.emin = r.rec_emin.as<int32_t>();
    ra.partA = r.partA.as<double>();
    ra.partT = r.partT.as<unsigned long long>();
    ra.tval = r.tval.as<unsigned long long>();
    ra.ploc = r.ploc.as<unsigned long long>();
    ra.parent = r.parent.as<int32_t>();
    ra.recA = r.rec_A.as<double>();
    ra.recT = r.rec_T.as<unsigned long long>();
    ra.reco = r.rec_o.as<uint32_t>();
    ra.counts = o.record_counts ? r.rec_counts.as<int32_t>() : nullptr;
    ra.stamp = r.rec_stamp.as<unsigned long long>();
    PA_CUDA(c, pa::launch_rs_min(ra, st));
    r.launches += 1;
    if (o.adaptive) {
        pa::AdaptArgs aa{};
        aa.E = r.E[cur].as<int32_t>();
        aa.emin = r.rec_emin.as<int32_t>();
        aa.R = r.R;
        aa.k = k;
        aa.J = o.adapt_J;
        aa.nmax = r.ad_nmax;
        aa.nch = r.nch;
        aa.rhoR = o.rho * (double)r.R;
        aa.delta = r.ad_delta;
        aa.qpow = r.d_qpow.as<double>();
        aa.part = r.ad_part.as<double>();
        aa.state = r.ad_state.as<int32_t>();
        aa.qsel = r.ad_qsel.as<int32_t>();
        aa.active = r.ad_active.as<int32_t>();
        aa.tidx = r.d_tidx.as<int32_t>();
        aa.jsel = r.rec_jsel.as<int32_t>();
        aa.beta = r.ad_beta.as<double>();
        aa.mode = o.adaptive;
        aa.accepts = r.rec_acc.as<unsigned long long>();
        const double attempts = (double)((int64_t)c->n * r.R * r.S);
        aa.acc_lo_n = o.acc_lo * attempts;
        aa.acc_hi_n = o.acc_hi * attempts;
        PA_CUDA(c, pa::launch_adapt(aa, st));
        r.launches += o.adaptive == 2 ? 1 : 2;
        ra.active = r.ad_active.as<int32_t>();
    }
    PA_CUDA(c, pa::launch_rs_rest(ra, st));
    r.launches += 2;

    pa::SweepArgs sa{};
    sa.g = g;
    sa.spins_in = r.spins[cur].as<int8_t>();
    sa.fields_in = r.fields[cur].as<int16_t>();
    sa.E_in = r.E[cur].as<int32_t>();
    sa.spins_out = r.spins[nxt].as<int8_t>();
    sa.fields_out = r.fields[nxt].as<int16_t>();
    sa.E_out = r.E[nxt].as<int32_t>();
    sa.parent = r.parent.as<int32_t>();
    sa.tables = r.d_tables.as<uint32_t>();
    sa.tidx = r.d_tidx.as<int32_t>();
    sa.active = o.adaptive ? r.ad_active.as<int32_t>() : nullptr;
    sa.R = r.R;
    sa.nblk = r.nblk;
    sa.S = r.S;
    sa.k = k;
    sa.key0 = k0;
    sa.key1 = k1;
    for (int r = 0; r < 10; ++r) {
        sa.rk0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        sa.rk1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    sa.best_rec = r.best_rec.as<int4>();
    sa.best_cfg = r.best_cfg.as<int8_t>();
    sa.accepts = r.rec_acc.as<unsigned long long>();
    sa.sweep_emin = r.rec_sweep.as<int32_t>();
    cudaEvent_t s0 = nullptr, s1 = nullptr;
    if (time_sweep) {
        PA_CUDA(c, cudaEventCreate(&s0));
        PA_CUDA(c, cudaEventCreate(&s1));
        r.ev_sweep.push_back(s0);
        r.ev_sweep.push_back(s1);
        PA_CUDA(c, cudaEventRecord(s0, st));
    }
    if (r.split) {   // fork: the tail words run on the second stream
        PA_CUDA(c, cudaEventRecord(r.ev_fork, st));
        PA_CUDA(c, cudaStreamWaitEvent(r.st2, r.ev_fork, 0));
        pa::SweepArgs sb = sa;
        sb.nblk = r.nblk2;
        sb.blk_base = r.blk_base2;
        PA_CUDA(c, pa::launch_sweep(r.sweep2, sb, r.st2));
        PA_CUDA(c, cudaEventRecord(r.ev_join, r.st2));
        r.launches += 1;
    }
    PA_CUDA(c, pa::launch_sweep(r.sweep, sa, st));
    if (r.split) PA_CUDA(c, cudaStreamWaitEvent(st, r.ev_join, 0));
    if (time_sweep) PA_CUDA(c, cudaEventRecord(s1, st));
    r.launches += 1;
    r.sweep_launches += 1;
    r.cur = nxt;
    if (o.nlm_period > 0 && k > 0 && k % o.nlm_period == 0) {
        pa::NlmArgs na{};
        na.g = g;
        na.pos = c->d_pos.as<int32_t>();
        na.spins = r.spins[nxt].as<int8_t>();
        const bool msc_run = r.variant == PA_VARIANT_MSC || r.variant == PA_VARIANT_MSC_PAIR;
        na.fields = msc_run ? nullptr : r.fields[nxt].as<int16_t>();   // multi-spin-coded sweeps read no fields
        na.E = r.E[nxt].as<int32_t>();
        na.R = r.R;
        na.k = k;
        na.key0 = k0;
        na.key1 = k1;
        na.active = o.adaptive ? r.ad_active.as<int32_t>() : nullptr;
        na.pairs = r.rec_nlm_pairs.as<int32_t>();
        na.flips = r.rec_nlm_flips.as<unsigned long long>();
        na.kind = o.nlm_kind;
        na.block = o.nlm_block;
        na.qrow = r.d_qblk.as<double>();
        na.tidx = r.d_tidx.as<int32_t>();
        int nl = 0;
        PA_CUDA(c, pa::launch_nonlocal(na, r.nlm_scratch.p, st, &nl));
        r.launches += nl;
    }
    return PA_OK;
}
}  // namespace

extern "C" {

int pa_anneal_run(pa_ctx *c, int32_t k_end) {
    if (!c) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "pa_anneal_begin has not run");
    if (k_end > r.K) k_end = r.K;
    if (k_end <= r.k_done) return PA_OK;
    cudaStream_t st = c->stream();
    cudaEvent_t e0, e1;
    PA_CUDA(c, cudaEventCreate(&e0));
    PA_CUDA(c, cudaEventCreate(&e1));
    r.ev_pending.push_back(e0);
    r.ev_pending.push_back(e1);
    PA_CUDA(c, cudaEventRecord(e0, st));
    // Adaptive runs: once the controller has reached beta_max every later step
    // is a no-op on the device. Enqueue in chunks of END_CHUNK steps, copy the
    // active flag of each chunk's last step to a pinned slot, and keep at most
    // END_WINDOW chunks ahead of the last flag read; a flag of 0 ends the loop
    // (the skipped steps count as done, exactly as if they had run). Not while
    // the stream is being captured, where the host may not wait.
    constexpr int32_t END_CHUNK = 32, END_WINDOW = 4;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    bool poll = r.opts.adaptive != 0 && cap == cudaStreamCaptureStatusNone;
    if (poll && !r.end_flag) {
        if (cudaHostAlloc(reinterpret_cast<void **>(&r.end_flag), 4 * END_WINDOW, cudaHostAllocDefault) != cudaSuccess) {
            r.end_flag = nullptr;
            poll = false;
        }
        for (int i = 0; poll && i < END_WINDOW; ++i)
            if (cudaEventCreateWithFlags(&r.end_ev[i], cudaEventDisableTiming) != cudaSuccess) poll = false;
        cudaGetLastError();
    }
    poll = poll && r.end_flag && r.end_ev[END_WINDOW - 1];
    int32_t chunk = 0;
    bool ended = false;
    for (int32_t k = r.k_done; k < k_end && !ended;) {
        const int32_t kc = poll ? std::min(k_end, k + END_CHUNK) : k_end;
        for (; k < kc; ++k)
            if (int rc = enqueue_step(c, k, st, r.opts.time_kernels != 0)) return rc;
        if (!poll || k >= k_end) break;
        const int slot = chunk % END_WINDOW;
        if (chunk >= END_WINDOW) {   // the slot's earlier copy: wait for it, then read it
            PA_CUDA(c, cudaEventSynchronize(r.end_ev[slot]));
            if (r.end_flag[slot] == 0) ended = true;
        }
        PA_CUDA(c, cudaMemcpyAsync(r.end_flag + slot, r.ad_active.as<int32_t>() + (k - 1), 4, cudaMemcpyDeviceToHost, st));
        PA_CUDA(c, cudaEventRecord(r.end_ev[slot], st));
        ++chunk;
    }
    PA_CUDA(c, pa::launch_stamp(r.rec_stamp.as<unsigned long long>() + k_end, st));
    r.launches += 1;
    PA_CUDA(c, cudaEventRecord(e1, st));
    r.k_done = k_end;
    return PA_OK;
}

int pa_sync(pa_ctx *c) {
    if (!c) return PA_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream());
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    collect_events(c->run);
    return PA_OK;
}

int pa_anneal(pa_ctx *c, const double *betas, int32_t K, int32_t R, int32_t sweeps, uint64_t seed,
              const pa_anneal_opts *opts) {
    int rc = pa_anneal_begin(c, betas, K, R, sweeps, seed, opts);
    if (rc) return rc;
    rc = pa_anneal_run(c, K);
    if (rc) return rc;
    return pa_sync(c);
}

}  // extern "C"

namespace {
// Lexicographic minimum of the per-block records; returns the block or -1.
int best_block(pa_ctx *c, int4 *rec) {
    RunState &r = c->run;
    std::vector<int4> br(r.nrec);
    if (copy(c, br.data(), r.best_rec.p, 16 * (size_t)r.nrec, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -2;
    }
    int best = -1;
    for (int b = 0; b < r.nrec; ++b) {
        if (br[b].y < 0) continue;
        if (best < 0) { best = b; continue; }
        const int4 &x = br[b], &y = br[best];
        if (x.x < y.x || (x.x == y.x && (x.y < y.y || (x.y == y.y && (x.z < y.z || (x.z == y.z && x.w < y.w))))))
            best = b;
    }
    if (best >= 0) *rec = br[best];
    return best;
}
}  // namespace

extern "C" {

int pa_batch_anneal(const pa_job *jobs, int32_t n_jobs, const pa_batch_opts *bopts, double *elapsed_ms) {
    if (!jobs || n_jobs < 1) return PA_EINVAL;
    pa_batch_opts bo{};
    if (bopts) bo = *bopts;
    int ns = bo.n_streams > 0 ? bo.n_streams : std::min<int>(n_jobs, 16);
    if (ns > 64) ns = 64;
    cudaStream_t origin = reinterpret_cast<cudaStream_t>(bo.stream);
    cudaStream_t own_origin = nullptr;   // the legacy default stream cannot be captured
    if (!origin && bo.use_graph) {
        if (cudaStreamCreateWithFlags(&own_origin, cudaStreamNonBlocking) != cudaSuccess) return PA_ECUDA;
        origin = own_origin;
    }
    std::vector<cudaStream_t> streams(ns, nullptr);
    std::vector<cudaEvent_t> joins(ns, nullptr);
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = PA_OK;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : joins) if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
        for (int j = 0; j < n_jobs; ++j)
            if (jobs[j].ctx) jobs[j].ctx->run.opts.stream = bo.stream;
        for (auto st : streams) if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
        if (own_origin) { cudaStreamSynchronize(own_origin); cudaStreamDestroy(own_origin); }
        cudaGetLastError();
    };
    auto cuda_err = [&](cudaError_t e, const char *where) {
        fail(jobs[0].ctx, PA_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
        return PA_ECUDA;
    };
    for (int i = 0; i < ns; ++i) {
        if (cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return PA_ECUDA;
        }
    }
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
        cleanup();
        return PA_ECUDA;
    }
    int32_t kmax = 0;
    for (int j = 0; j < n_jobs; ++j) {
        if (!jobs[j].ctx) { cleanup(); return PA_EINVAL; }
        pa_anneal_opts o = jobs[j].opts;
        o.stream = streams[j % ns];
        o.time_kernels = 0;
        rc = pa_anneal_begin(jobs[j].ctx, jobs[j].betas, jobs[j].K, jobs[j].R, jobs[j].sweeps, jobs[j].seed, &o);
        if (rc) { cleanup(); return rc; }
        kmax = std::max(kmax, jobs[j].K);
    }
    for (auto st : streams) cudaStreamSynchronize(st);
    if (cudaStreamSynchronize(origin) != cudaSuccess) { cleanup(); return PA_ECUDA; }
    const bool use_graph = bo.use_graph != 0;
    if (!use_graph) cudaEventRecord(t0, origin);
    if (use_graph) {
        cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            rc = cuda_err(e, "cudaStreamBeginCapture");
            cleanup();
            return rc;
        }
    }
    cudaEventRecord(fork, origin);
    for (auto st : streams) cudaStreamWaitEvent(st, fork, 0);
    for (int32_t k = 0; k < kmax && rc == PA_OK; ++k)
        for (int j = 0; j < n_jobs && rc == PA_OK; ++j)
            if (k < jobs[j].K) rc = enqueue_step(jobs[j].ctx, k, streams[j % ns], false);
    for (int j = 0; j < n_jobs && rc == PA_OK; ++j) {
        RunState &r = jobs[j].ctx->run;
        if (pa::launch_stamp(r.rec_stamp.as<unsigned long long>() + r.K, streams[j % ns]) != cudaSuccess) rc = PA_ECUDA;
        r.launches += 1;
        r.k_done = r.K;
    }
    for (int i = 0; i < ns; ++i) {
        cudaEventRecord(joins[i], streams[i]);
        cudaStreamWaitEvent(origin, joins[i], 0);
    }
    if (use_graph) {
        cudaError_t e = cudaStreamEndCapture(origin, &graph);
        if (rc == PA_OK && e != cudaSuccess) rc = cuda_err(e, "cudaStreamEndCapture");
        if (rc == PA_OK && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
            rc = cuda_err(e, "cudaGraphInstantiate");
        if (rc == PA_OK) {
            cudaEventRecord(t0, origin);
            if ((e = cudaGraphLaunch(exec, origin)) != cudaSuccess) rc = cuda_err(e, "cudaGraphLaunch");
        }
    }
    cudaEventRecord(t1, origin);
    if (cudaStreamSynchronize(origin) != cudaSuccess && rc == PA_OK) rc = PA_ECUDA;
    float ms = 0.f;
    if (rc == PA_OK && elapsed_ms && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess) *elapsed_ms = ms;
    cleanup();
    return rc;
}

int pa_best_record(pa_ctx *c, int32_t *energy, int32_t *step, int32_t *sweep, int32_t *slot) {
    if (!c) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "no anneal");
    if (int rc = pa_sync(c)) return rc;
    int4 rec;
    const int best = best_block(c, &rec);
    if (best == -2) return fail(c, PA_ECUDA, "best record copy failed");
    if (best < 0) return fail(c, PA_ESTATE, "no sweep has run");
    if (energy) *energy = rec.x;
    if (step) *step = rec.y;
    if (sweep) *sweep = rec.z;
    if (slot) *slot = rec.w;
    return PA_OK;
}

int pa_best(pa_ctx *c, int64_t *cut, int8_t *config, int32_t *step, int32_t *sweep) {
    if (!c) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "no anneal");
    if (int rc = pa_sync(c)) return rc;
    int4 rec;
    const int blk = best_block(c, &rec);
    if (blk == -2) return fail(c, PA_ECUDA, "best record copy failed");
    if (blk < 0) return fail(c, PA_ESTATE, "no sweep has run");
    if (step) *step = rec.y;
    if (sweep) *sweep = rec.z;
    if (cut) *cut = (c->W - (int64_t)rec.x) / 2;
    if (config) {
        std::vector<int8_t> cfg(c->np);
        PA_CUDA(c, copy(c, cfg.data(), r.best_cfg.as<int8_t>() + (size_t)blk * c->np, c->np,
                        cudaMemcpyDeviceToHost));
        for (int32_t i = 0; i < c->n; ++i) config[i] = cfg[c->pos[i]];
    }
    return PA_OK;
}

int pa_get_state(pa_ctx *c, int8_t *spins, int32_t *energies) {
    if (!c) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "no anneal");
    if (int rc = pa_sync(c)) return rc;
    if (spins) {
        std::vector<int8_t> buf((size_t)r.R * c->np);
        PA_CUDA(c, copy(c, buf.data(), r.spins[r.cur].p, buf.size(), cudaMemcpyDeviceToHost));
        for (int32_t s = 0; s < r.R; ++s)
            for (int32_t i = 0; i < c->n; ++i) spins[(size_t)s * c->n + i] = buf[(size_t)s * c->np + c->pos[i]];
    }
    if (energies)
        PA_CUDA(c, copy(c, energies, r.E[r.cur].p, 4 * (size_t)r.R, cudaMemcpyDeviceToHost));
    return PA_OK;
}

int pa_set_state(pa_ctx *c, const int8_t *spins, int32_t steps_done) {
    if (!c || !spins) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "pa_anneal_begin has not run");
    if (steps_done < 0 || steps_done > r.K) return fail(c, PA_EINVAL, "steps_done out of range");
    for (size_t t = 0; t < (size_t)r.R * c->n; ++t)
        if (spins[t] != 1 && spins[t] != -1) return fail(c, PA_EINVAL, "spins must be +1/-1");
    if (int rc = pa_sync(c)) return rc;
    std::vector<int8_t> buf((size_t)r.Rpad * c->np, 0);
    for (int32_t s = 0; s < r.Rpad; ++s) {
        const int32_t src = s < r.R ? s : r.R - 1;   // padding slots mirror the last replica
        for (int32_t i = 0; i < c->n; ++i) buf[(size_t)s * c->np + c->pos[i]] = spins[(size_t)src * c->n + i];
    }
    PA_CUDA(c, copy(c, r.spins[r.cur].p, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    PA_CUDA(c, pa::launch_fields(c->gdev(), r.spins[r.cur].as<int8_t>(), r.fields[r.cur].as<int16_t>(),
                                 r.E[r.cur].as<int32_t>(), r.Rpad, c->stream()));
    r.launches += 1;
    r.k_done = steps_done;
    return pa_sync(c);
}

int pa_energies(pa_ctx *c, const int8_t *spins, int32_t R, int32_t *energies, int64_t *cuts) {
    if (!c || R < 0) return PA_EINVAL;
    if (R == 0 || (!energies && !cuts)) return PA_OK;
    if (!spins) return PA_EINVAL;
    const size_t total = (size_t)R * c->n;
    for (size_t t = 0; t < total; ++t)
        if (spins[t] != 1 && spins[t] != -1) return fail(c, PA_EINVAL, "spins must be +1/-1");
    // Same kernel that builds the fields and energies of a population at the
    // start of an anneal; padding positions past n hold +1 and have no edges.
    std::vector<int8_t> buf((size_t)R * c->np, 1);
    for (int32_t s = 0; s < R; ++s)
        for (int32_t i = 0; i < c->n; ++i) buf[(size_t)s * c->np + c->pos[i]] = spins[(size_t)s * c->n + i];
    cudaStream_t st = c->stream();
    DevBuf dx, dh, dE;
    struct Drain {   // runs before the buffers are freed, on every return path
        cudaStream_t s;
        ~Drain() { cudaStreamSynchronize(s); }
    } drain{st};
    if (!dx.alloc(buf.size(), st) || !dh.alloc(2 * buf.size(), st) || !dE.alloc(4 * (size_t)R, st))
        return fail(c, PA_ENOMEM, "device allocation failed");
    std::vector<int32_t> E(R);
    PA_CUDA(c, copy(c, dx.p, buf.data(), buf.size(), cudaMemcpyHostToDevice, st, true));
    PA_CUDA(c, pa::launch_fields(c->gdev(), dx.as<int8_t>(), dh.as<int16_t>(), dE.as<int32_t>(), R, st));
    PA_CUDA(c, copy(c, E.data(), dE.p, 4 * (size_t)R, cudaMemcpyDeviceToHost, st, true));
    PA_CUDA(c, cudaStreamSynchronize(st));
    for (int32_t s = 0; s < R; ++s) {
        if (energies) energies[s] = E[s];
        if (cuts) cuts[s] = (c->W - (int64_t)E[s]) / 2;
    }
    return PA_OK;
}

int pa_run_info(pa_ctx *c, int32_t *R, int32_t *K, int32_t *sweeps, int32_t *steps_done) {
    if (!c) return PA_EINVAL;
    const RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "no anneal");
    if (R) *R = r.R;
    if (K) *K = r.K;
    if (sweeps) *sweeps = r.S;
    if (steps_done) *steps_done = r.k_done;
    return PA_OK;
}

int pa_stats(pa_ctx *c, pa_stats_t *out) {
    if (!c || !out) return PA_EINVAL;
    RunState &r = c->run;
    std::memset(out, 0, sizeof(*out));
    out->n_colours = c->ncol;
    out->max_degree = c->maxdeg;
    out->total_weight = c->W;
    out->h2d_bytes = c->h2d;
    out->d2h_bytes = c->d2h;
    if (!r.begun) return PA_OK;
    if (int rc = pa_sync(c)) return rc;
    int32_t steps = r.k_done;
    if (r.opts.adaptive && steps > 0) {
        std::vector<int32_t> act(steps);
        PA_CUDA(c, copy(c, act.data(), r.ad_active.p, 4 * (size_t)steps, cudaMemcpyDeviceToHost));
        int32_t s = 0;
        while (s < steps && act[s]) ++s;
        steps = s;
    }
    out->steps_run = steps;
    out->attempts = (int64_t)c->n * r.R * r.S * steps;
    if (steps > 0) {
        std::vector<unsigned long long> acc(steps);
        PA_CUDA(c, copy(c, acc.data(), r.rec_acc.p, 8 * (size_t)steps, cudaMemcpyDeviceToHost));
        for (auto v : acc) out->accepts += (int64_t)v;
    }
    out->kernel_launches = r.launches;
    out->sweep_launches = r.sweep_launches;
    out->variant = r.variant;
    out->anneal_ms = r.anneal_ms;
    out->sweep_ms = r.sweep_ms;
    out->h2d_bytes = c->h2d;
    out->d2h_bytes = c->d2h;
    // time to best: end of the step that recorded the final best
    int32_t E = 0, bstep = -1;
    if (steps > 0 && pa_best_record(c, &E, &bstep, nullptr, nullptr) == PA_OK && bstep >= 0) {
        std::vector<unsigned long long> st(r.k_done + 1);
        PA_CUDA(c, copy(c, st.data(), r.rec_stamp.p, 8 * (size_t)(r.k_done + 1), cudaMemcpyDeviceToHost));
        unsigned long long end = st[bstep + 1];
        if (end == 0 || end < st[0]) end = st[r.k_done];
        if (st[0] && end >= st[0]) out->t_best_ms = (double)(end - st[0]) * 1e-6;
    }
    return PA_OK;
}

int pa_step_stats(pa_ctx *c, pa_step_arrays *out) {
    if (!c || !out) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "no anneal");
    pa_stats_t st;
    if (int rc = pa_stats(c, &st)) return rc;
    const int32_t ks = st.steps_run;
    if (ks == 0) return PA_OK;
    std::vector<int32_t> emin(ks);
    std::vector<double> A(ks);
    PA_CUDA(c, copy(c, emin.data(), r.rec_emin.p, 4 * (size_t)ks, cudaMemcpyDeviceToHost));
    PA_CUDA(c, copy(c, A.data(), r.rec_A.p, 8 * (size_t)ks, cudaMemcpyDeviceToHost));
    std::vector<double> beta(ks);
    if (r.opts.adaptive || r.opts.reheat_after > 0)
        PA_CUDA(c, copy(c, beta.data(), r.ad_beta.p, 8 * (size_t)ks, cudaMemcpyDeviceToHost));
    else
        for (int32_t k = 0; k < ks; ++k) beta[k] = r.betas[k];
    if (out->beta) std::memcpy(out->beta, beta.data(), 8 * (size_t)ks);
    if (out->emin) std::memcpy(out->emin, emin.data(), 4 * (size_t)ks);
    if (out->A) std::memcpy(out->A, A.data(), 8 * (size_t)ks);
    if (out->T) PA_CUDA(c, copy(c, out->T, r.rec_T.p, 8 * (size_t)ks, cudaMemcpyDeviceToHost));
    if (out->o) PA_CUDA(c, copy(c, out->o, r.rec_o.p, 4 * (size_t)ks, cudaMemcpyDeviceToHost));
    if (out->accepts) PA_CUDA(c, copy(c, out->accepts, r.rec_acc.p, 8 * (size_t)ks, cudaMemcpyDeviceToHost));
    if (out->sweep_emin && r.S > 0)
        PA_CUDA(c, copy(c, out->sweep_emin, r.rec_sweep.p, 4 * (size_t)ks * r.S, cudaMemcpyDeviceToHost));
    if (out->nlm_pairs) PA_CUDA(c, copy(c, out->nlm_pairs, r.rec_nlm_pairs.p, 4 * (size_t)ks, cudaMemcpyDeviceToHost));
    if (out->nlm_flips) PA_CUDA(c, copy(c, out->nlm_flips, r.rec_nlm_flips.p, 8 * (size_t)ks, cudaMemcpyDeviceToHost));
    if (out->jsel) PA_CUDA(c, copy(c, out->jsel, r.rec_jsel.p, 4 * (size_t)ks, cudaMemcpyDeviceToHost));
    if (out->counts) {
        if (!r.opts.record_counts) return fail(c, PA_ESTATE, "record_counts was off");
        PA_CUDA(c, copy(c, out->counts, r.rec_counts.p, 4 * (size_t)ks * r.R, cudaMemcpyDeviceToHost));
    }
    if (out->t_ms) {
        std::vector<unsigned long long> sp(r.k_done + 1);
        PA_CUDA(c, copy(c, sp.data(), r.rec_stamp.p, 8 * (size_t)(r.k_done + 1), cudaMemcpyDeviceToHost));
        for (int32_t k = 0; k < ks; ++k)
            out->t_ms[k] = (sp[0] && sp[k + 1] >= sp[0]) ? (double)(sp[k + 1] - sp[0]) * 1e-6 : 0.0;
    }
    if (out->lnZ) {
        // ln Z(beta_k) = N ln 2 + sum_{j<=k} (-dbeta_j E_min,j + ln(A_j / R))
        double lnZ = (double)c->n * std::log(2.0), prev = 0.0;
        for (int32_t k = 0; k < ks; ++k) {
            const double dbeta = beta[k] - prev;
            lnZ += -dbeta * (double)emin[k] + std::log(A[k] / (double)r.R);
            out->lnZ[k] = lnZ;
            prev = beta[k];
        }
    }
    return PA_OK;
}

int pa_tables(pa_ctx *c, int32_t k, uint32_t *accept, double *qpow) {
    if (!c) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "no anneal");
    if (k < 0 || k >= r.ntables) return fail(c, PA_EINVAL, "table index out of range");
    if (accept) std::memcpy(accept, &r.tables[(size_t)k * (c->maxdeg + 1)], 4 * (size_t)(c->maxdeg + 1));
    if (qpow) {
        if (k >= r.nq) return fail(c, PA_EINVAL, "qpow index out of range");
        std::memcpy(qpow, &r.qpow[(size_t)k * 32], 8 * 32);
    }
    return PA_OK;
}

int pa_colouring(pa_ctx *c, int32_t *colour, int32_t *position) {
    if (!c) return PA_EINVAL;
    if (colour) std::memcpy(colour, c->colour.data(), 4 * (size_t)c->n);
    if (position) std::memcpy(position, c->pos.data(), 4 * (size_t)c->n);
    return c->ncol;
}

// ---------------------------------------------------------------- checkpoint
namespace {
struct CkptHeader {
    char magic[8];
    uint64_t graph_hash;
    int32_t n, R, K, S, k_done, adaptive;
    uint64_t seed;
    pa_anneal_opts opts;
    int32_t best[4];
};

// Device arrays that a checkpoint carries besides the population: the
// per-step records of the steps already run (so that statistics and curves
// continue across a resume) and, in adaptive mode, the controller's state.
struct RecSpec {
    DevBuf *buf;
    size_t per_step, extra;   // bytes = per_step * k_done + extra
};

std::vector<RecSpec> ckpt_records(RunState &r) {
    std::vector<RecSpec> v = {{&r.rec_emin, 4, 0},      {&r.rec_A, 8, 0},
                              {&r.rec_T, 8, 0},         {&r.rec_o, 4, 0},
                              {&r.rec_acc, 8, 0},       {&r.rec_sweep, 4 * (size_t)r.S, 0},
                              {&r.rec_stamp, 8, 8},     {&r.rec_nlm_pairs, 4, 0},
                              {&r.rec_nlm_flips, 8, 0}, {&r.rec_jsel, 4, 0}};
    if (r.opts.record_counts) v.push_back({&r.rec_counts, 4 * (size_t)r.R, 0});
    if (r.opts.adaptive) {
        v.push_back({&r.ad_state, 0, 16});
        v.push_back({&r.ad_qsel, 4, 0});
        v.push_back({&r.ad_active, 4, 0});
        v.push_back({&r.ad_beta, 8, 0});
        v.push_back({&r.d_tidx, 4, 0});
    }
    if (r.opts.reheat_after > 0) {
        v.push_back({&r.ad_state, 0, 16});
        v.push_back({&r.ad_qsel, 4, 0});
        v.push_back({&r.ad_beta, 8, 0});
        v.push_back({&r.d_tidx, 4, 0});
    }
    return v;
}
}  // namespace

int pa_save(pa_ctx *c, const char *path) {
    if (!c || !path) return PA_EINVAL;
    RunState &r = c->run;
    if (!r.begun) return fail(c, PA_ESTATE, "no anneal");
    CkptHeader h{};
    std::memcpy(h.magic, "PAMCCKP3", 8);
    h.graph_hash = c->graph_hash;
    h.n = c->n;
    h.R = r.R;
    h.K = r.K;
    h.S = r.S;
    h.k_done = r.k_done;
    h.adaptive = r.opts.adaptive;
    h.seed = r.seed;
    h.opts = r.opts;
    h.opts.stream = nullptr;
    h.best[1] = -1;
    std::vector<int8_t> cfg(c->n, 0);
    if (pa_best_record(c, &h.best[0], &h.best[1], &h.best[2], &h.best[3]) == PA_OK) {
        int64_t cut;
        pa_best(c, &cut, cfg.data(), nullptr, nullptr);
    }
    std::vector<int8_t> spins((size_t)r.R * c->n);
    if (int rc = pa_get_state(c, spins.data(), nullptr)) return rc;
    std::vector<std::vector<char>> recs;
    for (const RecSpec &rs : ckpt_records(r)) {
        recs.emplace_back(rs.per_step * (size_t)r.k_done + rs.extra);
        if (!recs.back().empty())
            PA_CUDA(c, copy(c, recs.back().data(), rs.buf->p, recs.back().size(), cudaMemcpyDeviceToHost));
    }
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(c, PA_EINVAL, "cannot open checkpoint for writing");
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    const int32_t nb = (int32_t)r.betas.size();
    ok = ok && std::fwrite(&nb, 4, 1, f) == 1;
    if (nb) ok = ok && std::fwrite(r.betas.data(), 8, nb, f) == (size_t)nb;
    ok = ok && std::fwrite(cfg.data(), 1, cfg.size(), f) == cfg.size();
    ok = ok && std::fwrite(spins.data(), 1, spins.size(), f) == spins.size();
    for (const auto &b : recs) ok = ok && (b.empty() || std::fwrite(b.data(), 1, b.size(), f) == b.size());
    std::fclose(f);
    return ok ? PA_OK : fail(c, PA_EINVAL, "checkpoint write failed");
}

int pa_load(pa_ctx *c, const char *path) {
    if (!c || !path) return PA_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(c, PA_EINVAL, "cannot open checkpoint");
    CkptHeader h{};
    int32_t nb = 0;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, "PAMCCKP3", 8) == 0 &&
              std::fread(&nb, 4, 1, f) == 1 && nb >= 0 && nb <= (1 << 26);
    if (!ok || h.graph_hash != c->graph_hash || h.n != c->n) {
        std::fclose(f);
        return fail(c, PA_EINVAL, "checkpoint does not match this graph");
    }
    std::vector<double> betas(nb);
    std::vector<int8_t> cfg(c->n), spins((size_t)h.R * c->n);
    ok = (nb == 0 || std::fread(betas.data(), 8, nb, f) == (size_t)nb) &&
         std::fread(cfg.data(), 1, cfg.size(), f) == cfg.size() &&
         std::fread(spins.data(), 1, spins.size(), f) == spins.size();
    if (!ok || h.k_done < 0 || h.k_done > h.K) {
        std::fclose(f);
        return fail(c, PA_EINVAL, "truncated checkpoint");
    }
    pa_anneal_opts o = h.opts;
    o.stream = c->run.opts.stream;
    int rc = pa_anneal_begin(c, nb ? betas.data() : nullptr, h.K, h.R, h.S, h.seed, &o);
    if (rc) {
        std::fclose(f);
        return rc;
    }
    const std::vector<RecSpec> specs = ckpt_records(c->run);
    std::vector<std::vector<char>> recs;
    for (const RecSpec &rs : specs) {
        recs.emplace_back(rs.per_step * (size_t)h.k_done + rs.extra);
        if (!recs.back().empty()) ok = ok && std::fread(recs.back().data(), 1, recs.back().size(), f) == recs.back().size();
    }
    std::fclose(f);
    if (!ok) return fail(c, PA_EINVAL, "truncated checkpoint");
    if ((rc = pa_sync(c))) return rc;   // the clears that pa_anneal_begin enqueued come first
    for (size_t i = 0; i < specs.size(); ++i)
        if (!recs[i].empty())
            PA_CUDA(c, copy(c, specs[i].buf->p, recs[i].data(), recs[i].size(), cudaMemcpyHostToDevice));
    if ((rc = pa_set_state(c, spins.data(), h.k_done))) return rc;
    if (h.best[1] >= 0) {
        // The restored best goes into the record of block 0 with its configuration; later
        // records only win if lexicographically smaller, as in an uninterrupted run.
        RunState &r = c->run;
        std::vector<int8_t> row(c->np, 0);
        for (int32_t i = 0; i < c->n; ++i) row[c->pos[i]] = cfg[i];
        const int4 br = make_int4(h.best[0], h.best[1], h.best[2], h.best[3]);
        PA_CUDA(c, copy(c, r.best_rec.p, &br, 16, cudaMemcpyHostToDevice));
        PA_CUDA(c, copy(c, r.best_cfg.p, row.data(), c->np, cudaMemcpyHostToDevice));
    }
    return PA_OK;
}

}  // extern "C"
