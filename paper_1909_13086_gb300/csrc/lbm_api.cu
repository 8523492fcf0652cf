// lbm_api.cu -- host side of the C ABI declared in include/lbm.h.
//
// Owns the device buffers of one lattice, derives the parameters (Eq. 5 for
// k1, Eq. 6 on request for k2, and the cavity unit mapping), and enqueues the
// sweep kernels on the handle's stream.  No torch types cross this boundary:
// a framework can lend its stream (cuda_stream) and its allocator
// (lbm_set_allocator).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

using namespace btrirt;

namespace {

thread_local char g_create_error[256] = "";

lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

constexpr int kDefaultRows = 1;       // rows walked by each thread of a block (tuned on GB300)
constexpr int kDefaultPrefetch = 16;  // L2 prefetch distance in rows (tuned on GB300)
// 16-bit storage is bound by instruction issue, and a thread's set-up (indices,
// the rounding seed, the block's tail) costs ~115 instructions against ~316
// per cell: 3 rows per thread spread it, with every row of a block prefetched
// (2048 x 1024 BF16-SR cavity on GB300, prefetch 8: 1 row 31.2 us, 2 rows
// 28.6, 3 rows 27.9, 4 rows 29.9, 6 rows 30.0 us per step; with the
// alternating sweep direction, 3 rows: prefetch 8 / 16 / 32 / 48 26.5 / 26.5 /
// 26.3 / 26.2 us).  FP32 is memory bound and fastest at 1 row (2 rows: +0.6
// us; prefetch 4 / 16 / 32: 41.8 / 41.5 / 41.4 us).
constexpr int kDefaultRows16 = 3;
constexpr int kDefaultPrefetch16 = 32;
constexpr int kDefaultGraphChunk = 128;  // longest graph-replayed piece (0 = direct launches)
constexpr int kGraphCache = 16;          // cached piece graphs per handle

// A piece of a step sequence: len sweeps from a given buffer parity, the last
// one diagnostic or not (every other sweep of a piece is plain).  Its graph is
// captured the second time the piece is asked for -- a one-off call never
// pays for a capture -- and replayed from then on.  exec == nullptr: seen
// once, not captured yet.
struct ChunkGraph {
    bool used = false;
    int parity = 0;
    int len = 0;
    bool diag = false;
    bool one_buffer = false;  // sweeps of one-buffer streaming, from phase `phase`
    int phase = 0;
    cudaGraphExec_t exec = nullptr;
    unsigned long long stamp = 0;
};

}  // namespace

struct lbm_s {
    int nx = 0, ny = 0, precision = LBM_FP32, device = 0;
    size_t esize = 4;           // bytes per population value
    int ntx = 0;                // column tiles of kTW cells
    int rows = kDefaultRows;    // rows per block
    int prefetch = kDefaultPrefetch;  // L2 prefetch distance in rows (0 = off)
    int graph_chunk = kDefaultGraphChunk;
    ChunkGraph graphs[kGraphCache];
    unsigned long long graph_clock = 0;
    lbm_launch_stats stats{};   // sweeps launched directly / replayed, graphs captured
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *buf[2] = {nullptr, nullptr};  // 18 planes each
    int cur = 0;                // buffer holding the current post-collision populations
    bool has_prev = false;      // buf[cur ^ 1] holds the previous step's populations
    // lbm_set_streaming: 1 = one-buffer streaming for all but the last one or
    // two sweeps of an lbm_step call; phase: 0 while buf[cur] holds the pull
    // layout (always between calls), 1 after a push sweep
    int streaming = LBM_STREAM_TWO_BUFFERS;  // set per precision by lbm_create
    int phase = 0;
    long long step = 0;
    long long diag_every = 0;
    bool params_set = false;
    lbm_params p{};
    lbm_derived d{};
    int lo2 = 0, hi2 = -1, strip_on = 0;
    dim3 block, grid;
    // staged sweep (16-bit storage): bands per tile column (-1: one wave of
    // blocks, 0: the row-per-block sweep), its grid and heated-wall partials
    int staged_mode = 0;
    int num_sms = 152;
    dim3 sgrid;
    int snq = 0;
    long long wait_limit = 1ll << 20;
    int force_timeout = 0;
    // scratch: reduction partials, tickets, record; allocated once
    void *scratch = nullptr;
    double *qpart = nullptr, *dpart = nullptr, *dpart2 = nullptr;
    unsigned *counters = nullptr;  // [0]: heated-wall ticket, [1]: diagnostics-fold ticket
    DevRecord *rec = nullptr;
    int nq = 0;
    // FP64 staging for field and population read-back / write (18 x nx*ny
    // doubles), allocated on first use
    double *stage = nullptr;
    // history ring (lbm_set_history): 4 doubles per entry
    double *hist = nullptr;
    long long hist_cap = 0;
    // allocator used for this handle's memory
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void *alloc_ctx = nullptr;
    char err[256] = "";
};

namespace {

int set_err(lbm_s *h, int code, const char *fmt, ...) {
    char *dst = h ? h->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(h, call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return set_err((h), LBM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// An NVTX range around a call, so that a profiler's timeline shows the steps
// the caller asked for (no cost unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void *dev_alloc(lbm_s *h, size_t bytes) {
    if (h->alloc) return h->alloc(bytes, h->alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lbm_s *h, void *p) {
    if (!p) return;
    if (h->release)
        h->release(p, h->alloc_ctx);
    else
        cudaFree(p);
}

size_t buffer_bytes(const lbm_s *h) {
    return (size_t)h->ntx * (size_t)h->ny * (size_t)kRS * h->esize;
}

// Resident blocks per SM of the staged sweep (128 threads, 64 registers,
// about 25 KB of shared memory each).
constexpr int kStagedBlocksPerSM = 8;

bool use_staged(const lbm_s *h) { return h->esize == 2 && h->staged_mode != 0; }

void set_grid(lbm_s *h) {
    h->block = dim3(kTW);
    h->grid = dim3(h->ntx, (h->ny + h->rows - 1) / h->rows);
    // blocks that fold the heated-wall inflow: the bottom row band of every
    // tile column (cavity) or the first tile column of every row band (Stefan)
    h->nq = h->p.problem == LBM_CAVITY ? (int)h->grid.x : (int)h->grid.y;
    // Staged sweep: bands of consecutive rows per tile column, as many as fill
    // the GPU with one wave of blocks, each band at least 4 rows high.
    int bands = h->staged_mode > 0 ? h->staged_mode
                                   : (h->num_sms * kStagedBlocksPerSM + h->ntx - 1) / h->ntx;
    bands = std::max(1, std::min(bands, std::max(1, h->ny / 4)));
    h->sgrid = dim3(h->ntx, bands);
    h->snq = h->p.problem == LBM_CAVITY ? (int)h->sgrid.x : (int)h->sgrid.y;
}

double *staging(lbm_s *h) {
    if (!h->stage)
        h->stage = static_cast<double *>(dev_alloc(h, (size_t)kPlanes * h->nx * h->ny * sizeof(double)));
    return h->stage;
}

template <typename real>
SweepArgs<real> make_args(const lbm_s *h, const void *src, void *dst) {
    SweepArgs<real> a{};
    a.src = src;
    a.dst = dst;
    a.nx = h->nx;
    a.ny = h->ny;
    a.ntx = h->ntx;
    a.rows = h->rows;
    a.prefetch = h->prefetch;
    a.parity = h->cur;
    a.k0 = (real)h->d.k0;
    a.k1 = (real)h->d.k1;
    a.k2 = (real)h->d.k2;
    a.k0f = (real)h->d.k0f;
    a.k1f = (real)h->d.k1f;
    a.k2f = (real)h->d.k2f;
    a.Lh = (real)h->d.Lh;
    a.inv_Lh = (real)(1.0 / h->d.Lh);
    a.gbeta = (real)h->d.gbeta;
    a.strip_on = h->strip_on;
    a.lo2 = h->lo2;
    a.hi2 = h->hi2;
    a.qpart = h->qpart;
    a.qcount = h->counters;
    a.nq = h->nq;
    a.dpart = h->dpart;
    a.dpart2 = h->dpart2;
    a.dticket = h->counters + 1;
    a.rec = h->rec;
    a.hist = h->hist;
    a.hist_cap = h->hist_cap;
    a.step = h->step;
    a.staged = 0;
    a.force_timeout = h->force_timeout;
    a.wait_limit = h->wait_limit;
    return a;
}

// Validate p and fill d (same mapping as documented in lbm.h).
int derive(lbm_s *h, const lbm_params *p, lbm_derived *d) {
    const double cs2 = 1.0 / 3.0, dT = 1.0;
    if (p->problem != LBM_CAVITY && p->problem != LBM_STEFAN)
        return set_err(h, LBM_ERR_ARG, "problem must be LBM_CAVITY or LBM_STEFAN");
    if (!(p->Ste > 0.0)) return set_err(h, LBM_ERR_ARG, "Ste must be > 0");
    if (!(p->alpha_override >= 0.0))
        return set_err(h, LBM_ERR_ARG, "alpha_override must be >= 0");
    std::memset(d, 0, sizeof(*d));
    d->Href = p->problem == LBM_CAVITY ? (double)h->ny : (double)h->nx;
    if (p->alpha_override > 0.0) {
        d->alpha = p->alpha_override;
        d->nu = (p->Pr > 0.0 ? p->Pr : 1.0) * d->alpha;
        d->gbeta = p->Ra > 0.0 ? p->Ra * d->nu * d->alpha / (dT * d->Href * d->Href * d->Href) : 0.0;
    } else {
        if (!(p->Ra > 0.0 && p->Pr > 0.0 && p->Ma > 0.0))
            return set_err(h, LBM_ERR_ARG, "Ra, Pr and Ma must be > 0 (or set alpha_override)");
        const double U = p->Ma * std::sqrt(cs2);
        d->nu = U * d->Href * std::sqrt(p->Pr / p->Ra);
        d->alpha = d->nu / p->Pr;
        d->gbeta = U * U / (dT * d->Href);
    }
    d->k1 = 1.0 / (d->alpha / cs2 + 0.5);  // Eq. 5, dt = 1
    d->k0 = p->k0;
    d->k2 = p->k2 < 0.0 ? 2.0 - d->k1 : p->k2;  // Eq. 6 on request
    d->k0f = p->k0f;
    d->k1f = p->k1f;
    d->k2f = 1.0 / (d->nu / cs2 + 0.5);
    d->Lh = dT / p->Ste;
    if (p->problem == LBM_CAVITY) {
        if (!(p->strip_width >= 0.0 && p->strip_center >= 0.0 && p->strip_center <= 1.0))
            return set_err(h, LBM_ERR_ARG, "strip centre must be in [0, 1] and width >= 0");
        d->a = h->nx * (p->strip_center - 0.5 * p->strip_width);
        d->b = h->nx * (p->strip_center + 0.5 * p->strip_width);
        d->heated_len = d->b - d->a;
    } else {
        d->heated_len = (double)h->ny;
    }
    const double ks[3] = {d->k0, d->k1, d->k2};
    for (double k : ks)
        if (!(k > 0.0 && k < 2.0))
            return set_err(h, LBM_ERR_ARG, "g rates k0, k1, k2 must lie in (0, 2) (k0=%g k1=%g k2=%g)",
                           d->k0, d->k1, d->k2);
    if (p->flow_on) {
        const double kf[3] = {d->k0f, d->k1f, d->k2f};
        for (double k : kf)
            if (!(k > 0.0 && k < 2.0))
                return set_err(h, LBM_ERR_ARG, "flow rates must lie in (0, 2) (k0f=%g k1f=%g k2f=%g)",
                               d->k0f, d->k1f, d->k2f);
    }
    if (!std::isfinite(p->init_amp)) return set_err(h, LBM_ERR_ARG, "init_amp must be finite");
    return LBM_OK;
}

// One sweep (plus the diagnostics fold after a diagnostic sweep), enqueued on
// the stream with programmatic serialization; advances the host's view of
// the state.
template <typename real, typename S>
int launch_one(lbm_s *h, bool diag) {
    const long long next = h->step + 1;
    SweepArgs<real> a = make_args<real>(h, h->buf[h->cur], h->buf[h->cur ^ 1]);
    a.step = next;
    const bool staged = use_staged(h);
    if (staged) {
        a.staged = 1;
        a.nq = h->snq;
    }
    cudaError_t e = launch_lattice<real, S>(a, h->p.problem, h->p.flow_on != 0, diag ? kSweepDiag : kSweep,
                                         staged ? h->sgrid : h->grid, h->block, h->stream, true);
    if (e != cudaSuccess) return set_err(h, LBM_ERR_CUDA, "sweep launch failed: %s", cudaGetErrorString(e));
    h->cur ^= 1;
    h->has_prev = true;
    h->step = next;
    return LBM_OK;
}

// One sweep of one-buffer streaming (Streaming in lbm_internal.h) in
// buf[cur]: the push sweep at phase 0, the local sweep at phase 1.  The parity
// word (rounding seed, sweep direction) alternates as it does over two
// buffers, so the populations are bitwise those of the pull sweeps.
template <typename real, typename S>
int launch_one_aa(lbm_s *h, bool diag) {
    const long long next = h->step + 1;
    SweepArgs<real> a = make_args<real>(h, h->buf[h->cur], h->buf[h->cur]);
    a.parity = h->cur ^ h->phase;
    a.step = next;
    cudaError_t e = launch_lattice<real, S>(a, h->p.problem, h->p.flow_on != 0, diag ? kSweepDiag : kSweep,
                                         h->grid, h->block, h->stream, true, h->phase ? kAALocal : kAAPush);
    if (e != cudaSuccess) return set_err(h, LBM_ERR_CUDA, "sweep launch failed: %s", cudaGetErrorString(e));
    h->phase ^= 1;
    h->has_prev = false;  // buf[cur ^ 1] is stale until the call's closing two-buffer sweeps
    h->step = next;
    return LBM_OK;
}

void drop_graphs(lbm_s *h) {
    for (ChunkGraph &g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = ChunkGraph();
    }
}

// Enqueues one piece: len sweeps, the last one diagnostic if diag.  Kernel
// arguments are fixed per piece -- the ping-pong pointers depend only on the
// starting parity -- and everything that changes from step to step (step
// counter, heated-wall sums, tickets, rounding seeds) lives in device memory,
// so a captured piece replays correctly at any later step.
template <typename real, typename S>
int run_piece(lbm_s *h, long long len, bool diag, bool one_buffer = false) {
    auto launch = [&](bool d) { return one_buffer ? launch_one_aa<real, S>(h, d) : launch_one<real, S>(h, d); };
    bool graphs = h->graph_chunk >= 2 && len >= 2 && len <= h->graph_chunk;
    if (graphs) {
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        graphs = cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone;
    }
    ChunkGraph *slot = nullptr;
    if (graphs) {
        for (ChunkGraph &g : h->graphs)
            if (g.used && g.parity == h->cur && g.len == len && g.diag == diag && g.one_buffer == one_buffer &&
                g.phase == h->phase)
                slot = &g;
        if (!slot) {  // first sighting: remember it, launch directly
            ChunkGraph *victim = &h->graphs[0];
            for (ChunkGraph &g : h->graphs) {
                if (!g.used) { victim = &g; break; }
                if (g.stamp < victim->stamp) victim = &g;
            }
            if (victim->exec) cudaGraphExecDestroy(victim->exec);
            *victim = ChunkGraph();
            victim->used = true;
            victim->parity = h->cur;
            victim->len = (int)len;
            victim->diag = diag;
            victim->one_buffer = one_buffer;
            victim->phase = h->phase;
            victim->stamp = ++h->graph_clock;
            graphs = false;
        } else if (!slot->exec) {  // second sighting: capture it
            const int cur0 = h->cur, phase0 = h->phase;
            const long long step0 = h->step;
            const bool prev0 = h->has_prev;
            CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            int rc = LBM_OK;
            for (long long j = 0; j < len && rc == LBM_OK; ++j) rc = launch(diag && j == len - 1);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
            h->cur = cur0;
            h->phase = phase0;
            h->step = step0;
            h->has_prev = prev0;
            if (rc != LBM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess)
                return set_err(h, LBM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess)
                return set_err(h, LBM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
            slot->exec = exec;
            h->stats.graphs_captured += 1;
        }
    }
    if (graphs) {
        slot->stamp = ++h->graph_clock;
        CUDA_TRY(h, cudaGraphLaunch(slot->exec, h->stream));
        if (one_buffer) {
            h->phase ^= (int)(len & 1);
            h->has_prev = false;
        } else {
            h->cur ^= (int)(len & 1);
            h->has_prev = true;
        }
        h->step += len;
        h->stats.sweeps_replayed += len;
        return LBM_OK;
    }
    for (long long j = 0; j < len; ++j) {
        const int rc = launch(diag && j == len - 1);
        if (rc != LBM_OK) return rc;
    }
    h->stats.sweeps_direct += len;
    return LBM_OK;
}

// n sweeps, cut into pieces that end at the diagnostic sweeps (every
// diag_every-th step and the call's last one) and are at most graph_chunk
// long: with diag_every = 100 every full piece is the same 100-sweep graph.
//
// With one-buffer streaming all but the last one or two sweeps of the call run
// in buf[cur] (an even number, so that the buffer holds the pull layout again),
// in pieces that end at the diagnostic steps; the closing sweeps run over the
// two buffers, so that between calls buf[cur ^ 1] holds the previous step's
// populations (the fields are recomputed from them) as with two buffers.
template <typename real, typename S>
int enqueue_steps(lbm_s *h, long long n) {
    long long aa = 0;
    if (h->streaming == LBM_STREAM_ONE_BUFFER && !use_staged(h) && n >= 3) aa = (n & 1) ? n - 1 : n - 2;
    for (long long done = 0; done < aa;) {
        long long len = aa - done;
        bool diag = false;
        if (h->diag_every > 0) {
            const long long k = h->diag_every - h->step % h->diag_every;
            if (k <= len) {
                len = k;
                diag = true;
            }
        }
        if (h->graph_chunk >= 2 && len > h->graph_chunk) {
            len = h->graph_chunk;
            diag = false;
        }
        const int rc = run_piece<real, S>(h, len, diag, true);
        if (rc != LBM_OK) return rc;
        done += len;
    }
    n -= aa;
    long long done = 0;
    while (done < n) {
        long long to_diag = n - done;  // sweeps up to and including the next diagnostic one
        if (h->diag_every > 0) {
            const long long k = h->diag_every - h->step % h->diag_every;
            if (k < to_diag) to_diag = k;
        }
        const bool full = h->graph_chunk >= 2 && to_diag > h->graph_chunk;
        const long long len = full ? h->graph_chunk : to_diag;
        const int rc = run_piece<real, S>(h, len, !full);
        if (rc != LBM_OK) return rc;
        done += len;
    }
    return LBM_OK;
}

template <typename real, typename S>
int enqueue_init(lbm_s *h) {
    SweepArgs<real> a = make_args<real>(h, nullptr, h->buf[h->cur]);
    a.aux = h->buf[h->cur ^ 1];
    a.step = 0;
    cudaError_t e = launch_init<real, S>(a, h->p.init_amp, (uint64_t)h->p.seed, h->grid, h->block,
                                      h->stream);
    if (e != cudaSuccess)
        return set_err(h, LBM_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(e));
    return LBM_OK;
}

template <typename real, typename S>
int enqueue_fields(lbm_s *h, double *out[6]) {
    cudaError_t e;
    if (h->step == 0 && !h->has_prev) {
        SweepArgs<real> a = make_args<real>(h, h->buf[h->cur], nullptr);
        a.oH = out[0]; a.oT = out[1]; a.oFL = out[2]; a.oUX = out[3]; a.oUY = out[4]; a.oRHO = out[5];
        e = launch_fields0<real, S>(a, h->p.flow_on != 0, h->grid, h->block, h->stream);
    } else {
        // Fields of step n are recomputed from the populations of step n-1,
        // which the ping-pong buffer still holds.
        SweepArgs<real> a = make_args<real>(h, h->buf[h->cur ^ 1], nullptr);
        a.oH = out[0]; a.oT = out[1]; a.oFL = out[2]; a.oUX = out[3]; a.oUY = out[4]; a.oRHO = out[5];
        e = launch_lattice<real, S>(a, h->p.problem, h->p.flow_on != 0, kFields, h->grid, h->block,
                                 h->stream, false);
    }
    if (e != cudaSuccess)
        return set_err(h, LBM_ERR_CUDA, "fields launch failed: %s", cudaGetErrorString(e));
    return LBM_OK;
}

template <typename real, typename S>
int repack(lbm_s *h, void *buf, void *buf2, bool to_staging) {
    cudaError_t e = launch_repack<S>(buf, buf2, h->stage, h->nx, h->ny, to_staging, h->stream);
    if (e != cudaSuccess) return set_err(h, LBM_ERR_CUDA, "repack launch failed: %s", cudaGetErrorString(e));
    return LBM_OK;
}

// Calls fn(Types<real, S>{}) for the handle's precision: the arithmetic type
// and the storage type of the populations.
template <typename R, typename S>
struct Types {
    using real = R;
    using store = S;
};
template <typename Fn>
int by_precision(int precision, Fn &&fn) {
    switch (precision) {
        case LBM_FP64: return fn(Types<double, double>{});
        case LBM_FP16: return fn(Types<float, F16<false>>{});
        case LBM_BF16: return fn(Types<float, BF16<false>>{});
        case LBM_FP16_SR: return fn(Types<float, F16<true>>{});
        case LBM_BF16_SR: return fn(Types<float, BF16<true>>{});
        default: return fn(Types<float, float>{});
    }
}
#define BTRIRT_T(t, F) F<typename decltype(t)::real, typename decltype(t)::store>

}  // namespace

extern "C" {

int lbm_create(int nx, int ny, int precision, void *cuda_stream, lbm_handle *out) {
    if (!out) return set_err(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 2 || ny < 2) return set_err(nullptr, LBM_ERR_ARG, "nx and ny must be >= 2");
    if (ny > 65535) return set_err(nullptr, LBM_ERR_ARG, "ny must be <= 65535");
    if ((long long)nx * ny > (1ll << 31))
        return set_err(nullptr, LBM_ERR_ARG, "lattice larger than 2^31 cells");
    if (precision < LBM_FP64 || precision > LBM_BF16_SR)
        return set_err(nullptr, LBM_ERR_ARG,
                       "precision must be LBM_FP64, LBM_FP32, LBM_FP16, LBM_BF16, LBM_FP16_SR or LBM_BF16_SR");
    lbm_s *h = new (std::nothrow) lbm_s();
    if (!h) return set_err(nullptr, LBM_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return set_err(nullptr, LBM_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    }
    h->nx = nx;
    h->ny = ny;
    h->precision = precision;
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        cudaGetLastError();
        h->num_sms = 152;
    }
    h->esize = precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2);
    h->ntx = (nx + kTW - 1) / kTW;
    if (h->esize == 2) {
        h->rows = kDefaultRows16;
        h->prefetch = kDefaultPrefetch16;
    }
    // One-buffer streaming where it pays: a step whose working set is one
    // buffer finds more of the previous step's rows in L2, and the local sweep
    // reads and writes aligned own slots (2048 x 1024 cavity on GB300: FP32
    // 41.4 -> 36.5 us per step, BF16-SR 26.1 -> 24.2, FP16-SR 26.5 -> 24.5).
    // FP64 is bound by its arithmetic (698 us per step either way).
    h->streaming = precision == LBM_FP64 ? LBM_STREAM_TWO_BUFFERS : LBM_STREAM_ONE_BUFFER;
    set_grid(h);
    h->alloc = g_alloc;
    h->release = g_free;
    h->alloc_ctx = g_alloc_ctx;
    if (cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return set_err(nullptr, LBM_ERR_CUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    // population buffers
    for (int b = 0; b < 2; ++b) {
        h->buf[b] = dev_alloc(h, buffer_bytes(h));
        if (!h->buf[b]) {
            lbm_destroy(h);
            return set_err(nullptr, LBM_ERR_OOM, "device allocation of %zu bytes failed",
                           buffer_bytes(h));
        }
    }
    // reduction scratch, carved from one allocation (each piece 256 B aligned):
    // counters | record | heated-wall partials | per-block diagnostics partials |
    // fold-kernel partials.
    // Sized for the largest grid any rows setting gives (one row per block).
    const size_t nblk = (size_t)h->ntx * (size_t)ny;
    const size_t nqmax = (size_t)(h->ntx > ny ? h->ntx : ny);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t nred = (nblk + 1023) / 1024;
    const size_t o_rec = 256, o_q = o_rec + up(sizeof(DevRecord)), o_d = o_q + up(nqmax * 8),
                 o_d2 = o_d + up(nblk * 32), bytes = o_d2 + up(nred * 32);
    h->scratch = dev_alloc(h, bytes);
    if (!h->scratch) {
        lbm_destroy(h);
        return set_err(nullptr, LBM_ERR_OOM, "device allocation of scratch failed");
    }
    char *s = static_cast<char *>(h->scratch);
    h->counters = reinterpret_cast<unsigned *>(s);
    h->rec = reinterpret_cast<DevRecord *>(s + o_rec);
    h->qpart = reinterpret_cast<double *>(s + o_q);
    h->dpart = reinterpret_cast<double *>(s + o_d);
    h->dpart2 = reinterpret_cast<double *>(s + o_d2);
    e = cudaMemsetAsync(h->scratch, 0, bytes, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        lbm_destroy(h);
        return set_err(nullptr, LBM_ERR_CUDA, "scratch clear failed: %s", cudaGetErrorString(e));
    }
    *out = h;
    return LBM_OK;
}

int lbm_set_params(lbm_handle h, const lbm_params *p) {
    if (!h || !p) return set_err(h, LBM_ERR_ARG, "NULL argument");
    DeviceGuard g(h->device);
    lbm_derived d;
    int rc = derive(h, p, &d);
    if (rc != LBM_OK) return rc;
    drop_graphs(h);
    h->p = *p;
    h->d = d;
    if (p->problem == LBM_CAVITY && p->strip_width > 0.0) {
        // crossing abscissa x_c heated iff a <= x_c <= b; 2 x_c is an integer
        h->lo2 = (int)std::ceil(2.0 * d.a);
        h->hi2 = (int)std::floor(2.0 * d.b);
        h->strip_on = 1;
    } else {
        h->lo2 = 0;
        h->hi2 = -1;
        h->strip_on = 0;
    }
    set_grid(h);
    h->step = 0;
    h->cur = 0;
    h->phase = 0;  // a call cut short mid-way through its one-buffer sweeps may have left 1
    h->has_prev = false;
    CUDA_TRY(h, cudaMemsetAsync(h->rec, 0, sizeof(DevRecord), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->counters, 0, 2 * sizeof(unsigned), h->stream));
    rc = by_precision(h->precision, [&](auto t) { return BTRIRT_T(t, enqueue_init)(h); });
    if (rc != LBM_OK) return rc;
    h->params_set = true;
    return LBM_OK;
}

int lbm_get_derived(lbm_handle h, lbm_derived *out) {
    if (!h || !out) return set_err(h, LBM_ERR_ARG, "NULL argument");
    if (!h->params_set) return set_err(h, LBM_ERR_STATE, "parameters not set");
    *out = h->d;
    return LBM_OK;
}

int lbm_step(lbm_handle h, long long n) {
    NvtxRange range("lbm_step");
    if (!h) return set_err(h, LBM_ERR_ARG, "NULL handle");
    if (n < 0) return set_err(h, LBM_ERR_ARG, "n must be >= 0");
    if (!h->params_set) return set_err(h, LBM_ERR_STATE, "parameters not set");
    if (n == 0) return LBM_OK;
    DeviceGuard g(h->device);
    return by_precision(h->precision, [&](auto t) { return BTRIRT_T(t, enqueue_steps)(h, n); });
}

int lbm_get_launch_stats(lbm_handle h, lbm_launch_stats *out) {
    if (!h || !out) return set_err(h, LBM_ERR_ARG, "NULL argument");
    *out = h->stats;
    return LBM_OK;
}

int lbm_set_diag_every(lbm_handle h, long long k) {
    if (!h || k < 0) return set_err(h, LBM_ERR_ARG, "bad argument");
    if (k != h->diag_every) drop_graphs(h);
    h->diag_every = k;
    return LBM_OK;
}

int lbm_read_fields(lbm_handle h, unsigned mask, double *H, double *T, double *fl, double *ux,
                    double *uy, double *rho) {
    if (!h) return set_err(h, LBM_ERR_ARG, "NULL handle");
    if (!h->params_set) return set_err(h, LBM_ERR_STATE, "parameters not set");
    if (h->step > 0 && !h->has_prev)
        return set_err(h, LBM_ERR_STATE, "no step taken since the populations were written");
    DeviceGuard g(h->device);
    const size_t P = (size_t)h->nx * h->ny;
    double *stage = staging(h);
    if (!stage) return set_err(h, LBM_ERR_OOM, "device allocation of the read-back staging failed");
    double *host[6] = {H, T, fl, ux, uy, rho};
    double *dev[6];
    for (int k = 0; k < 6; ++k) dev[k] = ((mask >> k) & 1u) && host[k] ? stage + k * P : nullptr;
    int rc = by_precision(h->precision, [&](auto t) { return BTRIRT_T(t, enqueue_fields)(h, dev); });
    if (rc != LBM_OK) return rc;
    for (int k = 0; k < 6; ++k)
        if (dev[k])
            CUDA_TRY(h, cudaMemcpyAsync(host[k], dev[k], P * sizeof(double), cudaMemcpyDeviceToHost,
                                        h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_diagnostics(lbm_handle h, lbm_diag *out) {
    if (!h || !out) return set_err(h, LBM_ERR_ARG, "NULL argument");
    if (!h->params_set) return set_err(h, LBM_ERR_STATE, "parameters not set");
    DeviceGuard g(h->device);
    DevRecord r;
    CUDA_TRY(h, cudaMemcpyAsync(&r, h->rec, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    // a timeout comes first: the sweep that ran out may not have reached the fold
    if (r.timeout != 0.0)
        return set_err(h, LBM_ERR_TIMEOUT,
                       "a bounded device wait of the staged sweep ran out; the populations since are not "
                       "valid (lbm_set_params or lbm_write_populations resets the state)");
    if (r.valid != 1.0 || (long long)r.step != h->step)
        return set_err(h, LBM_ERR_STATE, "no diagnostics for the current step");
    const double P = (double)h->nx * (double)h->ny;
    out->step = h->step;
    out->melt_fraction = r.melt_sum / P;
    out->H_total = r.H_sum;
    out->Q_strip = r.Q_last;
    out->Q_cum = r.Q_cum;
    out->Nu = h->d.heated_len > 0.0 ? r.Q_last * h->d.Href / (h->d.alpha * h->d.heated_len) : 0.0;
    out->front_x = r.melt_sum / (double)h->ny;
    out->max_u = r.max_u;
    out->nan_flag = r.nan_flag != 0.0 ? 1 : 0;
    if (out->nan_flag) return set_err(h, LBM_ERR_DIVERGED, "non-finite H or rho at step %lld", h->step);
    return LBM_OK;
}

int lbm_set_staging(lbm_handle h, int bands) {
    if (!h || bands < -1 || bands > 65535) return set_err(h, LBM_ERR_ARG, "bands must be -1, 0 or 1..65535");
    drop_graphs(h);
    h->staged_mode = bands;
    set_grid(h);
    return LBM_OK;
}

int lbm_set_streaming(lbm_handle h, int mode) {
    if (!h || (mode != LBM_STREAM_TWO_BUFFERS && mode != LBM_STREAM_ONE_BUFFER))
        return set_err(h, LBM_ERR_ARG, "mode must be LBM_STREAM_TWO_BUFFERS or LBM_STREAM_ONE_BUFFER");
    drop_graphs(h);
    h->streaming = mode;  // between calls buf[cur] always holds the pull layout (phase 0)
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_handle h, long long tries, int force_timeout) {
    if (!h || tries < 0 || (force_timeout != 0 && force_timeout != 1))
        return set_err(h, LBM_ERR_ARG, "tries must be >= 0 and force_timeout 0 or 1");
    drop_graphs(h);
    h->wait_limit = tries;
    h->force_timeout = force_timeout;
    return LBM_OK;
}

int lbm_read_populations(lbm_handle h, double *f, double *g, long long *step) {
    if (!h) return set_err(h, LBM_ERR_ARG, "NULL handle");
    if (!h->params_set) return set_err(h, LBM_ERR_STATE, "parameters not set");
    DeviceGuard gd(h->device);
    if (!staging(h)) return set_err(h, LBM_ERR_OOM, "device allocation of the staging failed");
    const size_t half = (size_t)9 * h->nx * h->ny;
    int rc = by_precision(h->precision,
                          [&](auto t) { return BTRIRT_T(t, repack)(h, h->buf[h->cur], nullptr, true); });
    if (rc != LBM_OK) return rc;
    if (f)
        CUDA_TRY(h, cudaMemcpyAsync(f, h->stage, half * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (g)
        CUDA_TRY(h, cudaMemcpyAsync(g, h->stage + half, half * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (step) *step = h->step;
    return LBM_OK;
}

int lbm_write_populations(lbm_handle h, const double *f, const double *g, long long step) {
    if (!h || !f || !g || step < 0) return set_err(h, LBM_ERR_ARG, "bad argument");
    if (!h->params_set) return set_err(h, LBM_ERR_STATE, "parameters not set");
    DeviceGuard gd(h->device);
    if (!staging(h)) return set_err(h, LBM_ERR_OOM, "device allocation of the staging failed");
    const size_t half = (size_t)9 * h->nx * h->ny;
    CUDA_TRY(h, cudaMemcpyAsync(h->stage, f, half * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->stage + half, g, half * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream));
    // With the flow off the f planes are never rewritten by a sweep, so both
    // buffers receive them.
    void *other = h->p.flow_on ? nullptr : h->buf[h->cur ^ 1];
    int rc = by_precision(h->precision,
                          [&](auto t) { return BTRIRT_T(t, repack)(h, h->buf[h->cur], other, false); });
    if (rc != LBM_OK) return rc;
    h->step = step;
    h->has_prev = false;
    h->phase = 0;  // the buffer now holds the pull layout
    CUDA_TRY(h, cudaMemsetAsync(h->rec, 0, sizeof(DevRecord), h->stream));
    // both tickets back to zero (a sweep cut short by a timeout may leave one taken)
    CUDA_TRY(h, cudaMemsetAsync(h->counters, 0, 2 * sizeof(unsigned), h->stream));
    const unsigned long long counter = (unsigned long long)step;
    CUDA_TRY(h, cudaMemcpyAsync(&h->rec->counter, &counter, sizeof(counter), cudaMemcpyHostToDevice,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_launch(lbm_handle h, int rows, int prefetch_rows, int graph_chunk) {
    if (!h || rows < 1 || rows > 1024 || prefetch_rows < 0 || graph_chunk < 0 || graph_chunk > 65536)
        return set_err(h, LBM_ERR_ARG,
                       "rows must be in [1, 1024], prefetch_rows >= 0, graph_chunk in [0, 65536]");
    drop_graphs(h);
    h->rows = rows;
    h->prefetch = prefetch_rows;
    h->graph_chunk = graph_chunk;
    set_grid(h);
    return LBM_OK;
}

int lbm_set_history(lbm_handle h, long long capacity) {
    if (!h || capacity < 0) return set_err(h, LBM_ERR_ARG, "lbm_set_history: bad argument");
    DeviceGuard g(h->device);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    dev_free(h, h->hist);
    h->hist = nullptr;
    h->hist_cap = 0;
    if (capacity == 0) return LBM_OK;
    h->hist = static_cast<double *>(dev_alloc(h, (size_t)capacity * 4 * sizeof(double)));
    if (!h->hist) return set_err(h, LBM_ERR_OOM, "lbm_set_history: device allocation failed");
    h->hist_cap = capacity;
    // all-ones bytes are NaN doubles: an empty slot has a NaN step
    CUDA_TRY(h, cudaMemsetAsync(h->hist, 0xff, (size_t)capacity * 4 * sizeof(double), h->stream));
    return LBM_OK;
}

int lbm_read_history(lbm_handle h, int max, long long *step, double *Q, double *Nu, double *melt,
                     int *count) {
    if (!h || max < 0 || !count) return set_err(h, LBM_ERR_ARG, "lbm_read_history: bad argument");
    *count = 0;
    if (!h->hist || max == 0) return LBM_OK;
    DeviceGuard g(h->device);
    std::vector<double> ring((size_t)h->hist_cap * 4);
    CUDA_TRY(h, cudaMemcpyAsync(ring.data(), h->hist, ring.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    // the newest entries, oldest first: slot of step s is s mod capacity
    const long long last = h->step;
    const long long first = std::max(0ll, std::max(last - h->hist_cap + 1, last - (long long)max + 1));
    int n = 0;
    for (long long s = first; s <= last; ++s) {
        const double *e = &ring[(size_t)(s % h->hist_cap) * 4];
        if (!(e[0] == (double)s)) continue;  // slot not written for step s (no heated wall, or not yet)
        if (step) step[n] = s;
        if (Q) Q[n] = e[1];
        if (Nu) Nu[n] = h->d.heated_len > 0.0 ? e[1] * h->d.Href / (h->d.alpha * h->d.heated_len) : 0.0;
        if (melt) melt[n] = e[2];
        ++n;
    }
    *count = n;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h) {
    if (!h) return LBM_OK;
    DeviceGuard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    dev_free(h, h->buf[0]);
    dev_free(h, h->buf[1]);
    dev_free(h, h->scratch);
    dev_free(h, h->stage);
    dev_free(h, h->hist);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return LBM_OK;
}

const char *lbm_last_error(lbm_handle h) { return h ? h->err : g_create_error; }

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return set_err(nullptr, LBM_ERR_ARG, "alloc and release must both be set or both NULL");
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return LBM_OK;
}

const char *lbm_version(void) { return "btrirt 0.1 sm_103a"; }

}  // extern "C"


// ---------------------------------------------------------------------------
// Autotuner: picks the launch shape (rows per block, L2 prefetch distance) for
// a lattice size by timing candidates on a scratch lattice of the same size,
// precision and parameters, so the caller's state is untouched.  Results are
// cached per (nx, ny, precision, problem, flow_on, streaming) for the process.
// ---------------------------------------------------------------------------
namespace {

struct TuneKey {
    int nx, ny, precision, problem, flow, streaming;
    bool operator==(const TuneKey &o) const {
        return nx == o.nx && ny == o.ny && precision == o.precision && problem == o.problem && flow == o.flow &&
               streaming == o.streaming;
    }
};
struct TuneEntry {
    TuneKey key;
    int rows, prefetch;
    float us_per_step;
};
std::mutex g_tune_mutex;
std::vector<TuneEntry> g_tune_cache;

}  // namespace

extern "C" int lbm_autotune(lbm_handle h, int steps_per_trial, int *rows_out, int *prefetch_out,
                            float *us_per_step_out) {
    if (!h || steps_per_trial < 1) return set_err(h, LBM_ERR_ARG, "lbm_autotune: bad argument");
    if (!h->params_set) return set_err(h, LBM_ERR_STATE, "lbm_autotune: parameters not set");
    const TuneKey key{h->nx, h->ny, h->precision, h->p.problem, h->p.flow_on != 0, h->streaming};
    TuneEntry best{key, h->rows, h->prefetch, 0.0f};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (const TuneEntry &e : g_tune_cache)
            if (e.key == key) {
                best = e;
                cached = true;
            }
    }
    if (!cached) {
        DeviceGuard g(h->device);
        lbm_handle t = nullptr;
        int rc = lbm_create(h->nx, h->ny, h->precision, h->stream, &t);
        if (rc != LBM_OK) return set_err(h, rc, "lbm_autotune: scratch lattice: %s", lbm_last_error(nullptr));
        rc = lbm_set_params(t, &h->p);
        if (rc == LBM_OK) rc = lbm_set_streaming(t, h->streaming);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (rc == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
            rc = set_err(h, LBM_ERR_CUDA, "lbm_autotune: cudaEventCreate failed");
        best.us_per_step = 1e30f;
        const int rows_c[] = {1, 2, 3, 4};
        const int pf_c[] = {0, 2, 4, 8, 16, 24, 32, 48};
        for (int rows : rows_c) {
            if (rc != LBM_OK || rows > h->ny) break;
            for (int pf : pf_c) {
                if (rc != LBM_OK) break;
                if (pf >= h->ny) continue;
                rc = lbm_set_launch(t, rows, pf, h->graph_chunk);
                if (rc == LBM_OK) rc = lbm_step(t, 4);  // warm-up (and graph capture)
                float best_ms = 1e30f;
                for (int rep = 0; rep < 2 && rc == LBM_OK; ++rep) {
                    if (cudaEventRecord(e0, t->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
                    if (rc == LBM_OK) rc = lbm_step(t, steps_per_trial);
                    if (rc == LBM_OK && (cudaEventRecord(e1, t->stream) != cudaSuccess ||
                                         cudaEventSynchronize(e1) != cudaSuccess))
                        rc = LBM_ERR_CUDA;
                    float ms = 0.0f;
                    if (rc == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms)
                        best_ms = ms;
                }
                const float us = best_ms * 1000.0f / (float)steps_per_trial;
                if (rc == LBM_OK && us < best.us_per_step) {
                    best.rows = rows;
                    best.prefetch = pf;
                    best.us_per_step = us;
                }
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        lbm_destroy(t);
        if (rc != LBM_OK) return set_err(h, rc < 0 ? rc : LBM_ERR_CUDA, "lbm_autotune: trial failed");
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache.push_back(best);
    }
    const int rc = lbm_set_launch(h, best.rows, best.prefetch, h->graph_chunk);
    if (rc != LBM_OK) return rc;
    if (rows_out) *rows_out = best.rows;
    if (prefetch_out) *prefetch_out = best.prefetch;
    if (us_per_step_out) *us_per_step_out = cached ? 0.0f : best.us_per_step;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batches: many lattices advanced by one launch per step.
// ---------------------------------------------------------------------------
struct lbm_batch_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int max = 0;
    std::vector<lbm_s *> members;
    void *entries = nullptr;  // device table: max BatchEntry<real>
    int *parity = nullptr;    // device: source buffer of each member
    int *starts = nullptr;    // device: first block of each member
    std::vector<unsigned char> host_entries;
    std::vector<int> host_starts;
    std::vector<int> host_parity;
    int nblocks = 0;
    int uniform = 0;          // blocks per member when all members have the same count
    int rows = 0;             // launch shape: rows per block (0: 2, or 4 with 16-bit storage),
    int prefetch = -1;        // L2 prefetch distance (-1: 4 rows),
    int interleave = 1;       // interleaved block order (uniform batches only; see batch_kernel)
    int streaming = -1;       // lbm_batch_set_streaming; -1: one buffer, two for FP64
    bool dirty = true;        // table must be rebuilt and uploaded
    int precision = -1, problem = -1, flow = -1;
    int graph_chunk = 128;    // longest graph-replayed piece; even, so that every
                              // piece starts at an even step of the call
    ChunkGraph graphs[kGraphCache];  // pieces as for a single lattice (parity unused:
                                     // the members' parities are a device table)
    unsigned long long graph_clock = 0;
    cudaEvent_t ev = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void *alloc_ctx = nullptr;
};

namespace {

int batch_err(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_error, sizeof(g_create_error), fmt, ap);
    va_end(ap);
    return code;
}

#define BATCH_TRY(call)                                                                         \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return batch_err(LBM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void batch_free(lbm_batch_s *b, void *p) {
    if (!p) return;
    if (b->release) b->release(p, b->alloc_ctx); else cudaFree(p);
}

void batch_drop_graph(lbm_batch_s *b) {
    for (ChunkGraph &g : b->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = ChunkGraph();
    }
}

template <typename real>
size_t entry_bytes() { return sizeof(BatchEntry<real>); }

// Default launch shape of a batch, whatever the members' own lbm_set_launch
// settings: 2 rows per block (4 with 16-bit storage), L2 prefetch 4 rows
// ahead, blocks of a one-size batch interleaved over the members -- the
// fastest shapes for 64 cavities of 256 x 128 on GB300 (FP32 46.1 us per
// step, 55.9 with 2 rows member by member and no alternating direction;
// BF16-SR 32.1 us, 43.3).  Longer prefetch distances run ahead of a small
// member's sweep (FP32, 2 rows: prefetch 4 / 8 / 16 / 32 46.1 / 47.4 / 51.5 /
// 57.5 us).  Results do not depend on it.
constexpr int kBatchRows32 = 2, kBatchRows16 = 4, kBatchPrefetch32 = 4, kBatchPrefetch16 = 4;

template <typename real>
void batch_build(lbm_batch_s *b) {
    const size_t eb = entry_bytes<real>();
    b->host_entries.assign(eb * b->members.size(), 0);
    b->host_starts.assign(b->members.size(), 0);
    b->uniform = 0;
    int start = 0;
    for (size_t r = 0; r < b->members.size(); ++r) {
        lbm_s *h = b->members[r];
        const int rows = b->rows > 0 ? b->rows : (h->esize == 2 ? kBatchRows16 : kBatchRows32);
        const int gy = (h->ny + rows - 1) / rows;
        BatchEntry<real> e{};
        for (int p = 0; p < 2; ++p) {
            e.a[p] = make_args<real>(h, h->buf[p], h->buf[p ^ 1]);
            e.a[p].parity = p;
            e.a[p].rows = rows;
            e.a[p].prefetch = b->prefetch >= 0 ? b->prefetch : (h->esize == 2 ? kBatchPrefetch16 : kBatchPrefetch32);
            e.a[p].nq = h->p.problem == LBM_CAVITY ? (int)h->grid.x : gy;
        }
        e.start = start;
        b->host_starts[r] = start;
        e.gx = (int)h->grid.x;
        e.gy = gy;
        const int nb = e.gx * e.gy;
        b->uniform = r == 0 ? nb : (b->uniform == nb ? nb : 0);
        start += e.gx * e.gy;
        std::memcpy(b->host_entries.data() + r * eb, &e, eb);
    }
    b->nblocks = start;
}

template <typename real, typename S>
int batch_steps(lbm_batch_s *b, long long n) {
    const int nm = (int)b->members.size();
    if (b->dirty) {
        batch_build<real>(b);
        BATCH_TRY(cudaMemcpyAsync(b->entries, b->host_entries.data(), b->host_entries.size(),
                                  cudaMemcpyHostToDevice, b->stream));
        BATCH_TRY(cudaMemcpyAsync(b->starts, b->host_starts.data(), b->host_starts.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, b->stream));
        batch_drop_graph(b);
        b->dirty = false;
    }
    b->host_parity.resize(nm);
    for (int r = 0; r < nm; ++r) b->host_parity[r] = b->members[r]->cur;
    BATCH_TRY(cudaMemcpyAsync(b->parity, b->host_parity.data(), nm * sizeof(int), cudaMemcpyHostToDevice,
                              b->stream));
    // Pieces: graph_chunk plain sweeps while more than that remain, then the
    // rest, ending with the diagnostic sweep.  Step j of a piece uses buffer
    // parity parity[r] ^ (j & 1); pieces start at even steps of the call, so
    // a captured piece replays anywhere.  As for a single lattice, a piece's
    // graph is captured the second time it is asked for.
    long long done = 0;
    const int K = b->graph_chunk;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    BATCH_TRY(cudaStreamIsCapturing(b->stream, &st));
    const bool capturing = st != cudaStreamCaptureStatusNone;
    // One-buffer streaming (lbm_batch_set_streaming): the first sweeps of the
    // call, an even number, alternate push (even j) and local (odd j) sweeps
    // in each member's buffer parity[r]; the last one or two run over the two
    // buffers, so that between calls every member's state is the two-buffer one.
    const bool one = b->streaming < 0 ? b->precision != LBM_FP64 : b->streaming == LBM_STREAM_ONE_BUFFER;
    const long long aa = (one && n >= 3) ? ((n & 1) ? n - 1 : n - 2) : 0;
    auto direct = [&](long long from, long long len, bool diag, bool ob) -> int {
        for (long long j = 0; j < len; ++j) {
            const long long jj = from + j;
            const int sm = ob ? ((jj & 1) ? kAALocal : kAAPush) : kPull;
            const cudaError_t e = launch_batch<real, S>(b->entries, b->starts, b->parity, nm, b->uniform,
                                                        b->uniform > 0 ? b->interleave : 0, b->nblocks,
                                                        b->problem, b->flow != 0,
                                                        diag && j == len - 1, (int)(jj & 1),
                                                        b->stream, true, sm);
            if (e != cudaSuccess) return batch_err(LBM_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
        }
        return LBM_OK;
    };
    // One piece, starting at an even step `from` of the call: launched
    // directly the first time it is asked for, captured the second time,
    // replayed from then on.
    auto piece = [&](long long from, long long len, bool diag, bool ob) -> int {
        ChunkGraph *slot = nullptr;
        const bool graphs = K >= 2 && len >= 2 && len <= K && !capturing;
        if (graphs) {
            for (ChunkGraph &g : b->graphs)
                if (g.used && g.len == len && g.diag == diag && g.one_buffer == ob) slot = &g;
            if (!slot) {
                ChunkGraph *victim = &b->graphs[0];
                for (ChunkGraph &g : b->graphs) {
                    if (!g.used) { victim = &g; break; }
                    if (g.stamp < victim->stamp) victim = &g;
                }
                if (victim->exec) cudaGraphExecDestroy(victim->exec);
                *victim = ChunkGraph();
                victim->used = true;
                victim->len = (int)len;
                victim->diag = diag;
                victim->one_buffer = ob;
                victim->stamp = ++b->graph_clock;
            } else if (!slot->exec) {
                BATCH_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                const int rc = direct(0, len, diag, ob);
                cudaGraph_t g = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                if (rc != LBM_OK || e2 != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return rc != LBM_OK ? rc
                                        : batch_err(LBM_ERR_CUDA, "batch graph capture failed: %s",
                                                    cudaGetErrorString(e2));
                }
                const cudaError_t e3 = cudaGraphInstantiate(&slot->exec, g, 0);
                cudaGraphDestroy(g);
                if (e3 != cudaSuccess) {
                    slot->exec = nullptr;
                    return batch_err(LBM_ERR_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e3));
                }
            }
        }
        if (slot && slot->exec) {
            slot->stamp = ++b->graph_clock;
            BATCH_TRY(cudaGraphLaunch(slot->exec, b->stream));
            return LBM_OK;
        }
        return direct(from, len, diag, ob);
    };
    while (done < aa) {  // K and aa are even: every piece starts at an even step
        const long long len = (K >= 2 && aa - done > K) ? K : aa - done;
        const int rc = piece(done, len, false, true);
        if (rc != LBM_OK) return rc;
        done += len;
    }
    while (done < n) {
        const bool full = K >= 2 && n - done > K;
        const long long len = full ? K : n - done;
        const int rc = piece(done, len, !full, false);
        if (rc != LBM_OK) return rc;
        done += len;
    }
    for (lbm_s *h : b->members) {
        h->step += n;
        h->cur ^= (int)(n & 1);
        h->has_prev = true;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int max_lattices, void *cuda_stream, lbm_batch *out) {
    if (!out || max_lattices < 1 || max_lattices > 65536)
        return batch_err(LBM_ERR_ARG, "lbm_batch_create: need out != NULL and 1 <= max_lattices <= 65536");
    *out = nullptr;
    lbm_batch_s *b = new (std::nothrow) lbm_batch_s();
    if (!b) return batch_err(LBM_ERR_OOM, "host allocation failed");
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return batch_err(LBM_ERR_CUDA, "cudaGetDevice failed");
    }
    b->max = max_lattices;
    b->alloc = g_alloc;
    b->release = g_free;
    b->alloc_ctx = g_alloc_ctx;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    const size_t table = ((size_t)max_lattices * sizeof(BatchEntry<double>) + 255) / 256 * 256;
    const size_t bytes = table + 2 * (size_t)max_lattices * sizeof(int);
    void *mem = nullptr;
    if (e == cudaSuccess) {
        if (b->alloc) {
            mem = b->alloc(bytes, b->alloc_ctx);
        } else if (cudaMalloc(&mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            mem = nullptr;
        }
    }
    if (e != cudaSuccess || !mem) {
        lbm_batch_destroy(b);
        return batch_err(e != cudaSuccess ? LBM_ERR_CUDA : LBM_ERR_OOM, "lbm_batch_create: setup failed");
    }
    b->entries = mem;
    b->parity = reinterpret_cast<int *>(static_cast<char *>(mem) + table);
    b->starts = b->parity + max_lattices;
    *out = b;
    return LBM_OK;
}

int lbm_batch_add(lbm_batch b, lbm_handle h) {
    if (!b || !h) return batch_err(LBM_ERR_ARG, "lbm_batch_add: NULL argument");
    if (!h->params_set) return batch_err(LBM_ERR_STATE, "lbm_batch_add: lattice has no parameters");
    if (h->device != b->device) return batch_err(LBM_ERR_ARG, "lbm_batch_add: lattice on another device");
    for (lbm_s *m : b->members)
        if (m == h) return batch_err(LBM_ERR_ARG, "lbm_batch_add: lattice already in the batch");
    if ((int)b->members.size() >= b->max) return batch_err(LBM_ERR_ARG, "lbm_batch_add: batch is full");
    if (!b->members.empty() &&
        (h->precision != b->precision || h->p.problem != b->problem || (h->p.flow_on != 0) != (b->flow != 0)))
        return batch_err(LBM_ERR_ARG,
                         "lbm_batch_add: every lattice of a batch needs the same precision, problem and flow_on");
    if (b->members.empty()) {
        b->precision = h->precision;
        b->problem = h->p.problem;
        b->flow = h->p.flow_on != 0;
    }
    b->members.push_back(h);
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_remove(lbm_batch b, lbm_handle h) {
    if (!b || !h) return batch_err(LBM_ERR_ARG, "lbm_batch_remove: NULL argument");
    for (size_t r = 0; r < b->members.size(); ++r) {
        if (b->members[r] == h) {
            // work queued by the batch on this lattice must finish before the
            // caller uses it on its own stream
            DeviceGuard g(b->device);
            BATCH_TRY(cudaEventRecord(b->ev, b->stream));
            BATCH_TRY(cudaStreamWaitEvent(h->stream, b->ev, 0));
            b->members.erase(b->members.begin() + (long)r);
            b->dirty = true;
            return LBM_OK;
        }
    }
    return batch_err(LBM_ERR_ARG, "lbm_batch_remove: lattice not in the batch");
}

int lbm_batch_count(lbm_batch b, int *count) {
    if (!b || !count) return batch_err(LBM_ERR_ARG, "lbm_batch_count: NULL argument");
    *count = (int)b->members.size();
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, long long n) {
    NvtxRange range("lbm_batch_step");
    if (!b || n < 0) return batch_err(LBM_ERR_ARG, "lbm_batch_step: bad argument");
    if (n == 0 || b->members.empty()) return LBM_OK;
    DeviceGuard g(b->device);
    // order the batch after everything already queued on the members' streams
    cudaStream_t last = nullptr;
    for (lbm_s *h : b->members) {
        if (h->stream == b->stream || h->stream == last) continue;
        BATCH_TRY(cudaEventRecord(b->ev, h->stream));
        BATCH_TRY(cudaStreamWaitEvent(b->stream, b->ev, 0));
        last = h->stream;
    }
    const int rc = by_precision(b->precision, [&](auto t) { return BTRIRT_T(t, batch_steps)(b, n); });
    if (rc != LBM_OK) return rc;
    // and the members' streams after the batch
    BATCH_TRY(cudaEventRecord(b->ev, b->stream));
    last = nullptr;
    for (lbm_s *h : b->members) {
        if (h->stream == b->stream || h->stream == last) continue;
        BATCH_TRY(cudaStreamWaitEvent(h->stream, b->ev, 0));
        last = h->stream;
    }
    return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch b, int rows_per_block, int prefetch_rows, int interleave) {
    if (!b || rows_per_block < 0 || rows_per_block > 1024 || prefetch_rows < -1 || (interleave != 0 && interleave != 1))
        return batch_err(LBM_ERR_ARG,
                         "lbm_batch_set_launch: rows in [0, 1024], prefetch_rows >= -1, interleave 0 or 1");
    b->rows = rows_per_block;
    b->prefetch = prefetch_rows;
    b->interleave = interleave;
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_set_streaming(lbm_batch b, int mode) {
    if (!b || (mode != LBM_STREAM_TWO_BUFFERS && mode != LBM_STREAM_ONE_BUFFER))
        return batch_err(LBM_ERR_ARG,
                         "lbm_batch_set_streaming: mode must be LBM_STREAM_TWO_BUFFERS or LBM_STREAM_ONE_BUFFER");
    if (b->stream) cudaStreamSynchronize(b->stream);  // no captured piece may be in flight
    batch_drop_graph(b);
    b->streaming = mode;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b) {
    if (!b) return LBM_OK;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    batch_free(b, b->entries);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch autotuner: times launch shapes of a batch (rows per block, L2
// prefetch distance, interleaved block order) on scratch lattices of the same
// composition and applies the fastest; cached per composition for the
// process.
// ---------------------------------------------------------------------------
namespace {

struct BatchTune {
    std::string key;
    int rows, prefetch, interleave;
    float us_per_step;
};
std::mutex g_btune_mutex;
std::vector<BatchTune> g_btune_cache;

// The composition: precision, problem, flow, streaming, then every member's
// size in order.
std::string batch_key(const lbm_batch_s *b) {
    std::string k = std::to_string(b->precision) + "/" + std::to_string(b->problem) + "/" +
                    std::to_string(b->flow) + "/" + std::to_string(b->streaming);
    for (const lbm_s *h : b->members) k += "|" + std::to_string(h->nx) + "x" + std::to_string(h->ny);
    return k;
}

}  // namespace

extern "C" int lbm_batch_autotune(lbm_batch b, int steps_per_trial, int *rows_out, int *prefetch_out,
                                  int *interleave_out, float *us_per_step_out) {
    if (!b || steps_per_trial < 1) return batch_err(LBM_ERR_ARG, "lbm_batch_autotune: bad argument");
    if (b->members.empty()) return batch_err(LBM_ERR_STATE, "lbm_batch_autotune: the batch is empty");
    const std::string key = batch_key(b);
    BatchTune best{key, b->rows, b->prefetch, b->interleave, 0.0f};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_btune_mutex);
        for (const BatchTune &e : g_btune_cache)
            if (e.key == key) {
                best = e;
                cached = true;
            }
    }
    if (!cached) {
        DeviceGuard g(b->device);
        // scratch lattices of the same sizes and parameters, in a scratch batch
        // on the batch's stream: the members' states are not touched
        std::vector<lbm_handle> scratch;
        lbm_batch t = nullptr;
        int rc = lbm_batch_create((int)b->members.size(), b->stream, &t);
        if (rc == LBM_OK) t->streaming = b->streaming;
        for (size_t r = 0; r < b->members.size() && rc == LBM_OK; ++r) {
            const lbm_s *h = b->members[r];
            lbm_handle s = nullptr;
            rc = lbm_create(h->nx, h->ny, h->precision, b->stream, &s);
            if (rc == LBM_OK) {
                scratch.push_back(s);
                rc = lbm_set_params(s, &h->p);
            }
            if (rc == LBM_OK) rc = lbm_batch_add(t, s);
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (rc == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
            rc = LBM_ERR_CUDA;
        const int rows_c[] = {1, 2, 3, 4};
        const int pf_c[] = {0, 4, 8, 16};
        const int ninter = b->members.size() > 1 ? 2 : 1;  // interleaving needs several members
        best.us_per_step = 1e30f;
        for (int rows : rows_c) {
            for (int k = 0; k < 4 && rc == LBM_OK; ++k) {
                for (int il = 0; il < ninter && rc == LBM_OK; ++il) {
                    rc = lbm_batch_set_launch(t, rows, pf_c[k], il);
                    if (rc == LBM_OK) rc = lbm_batch_step(t, 4);  // warm-up, table upload
                    if (rc == LBM_OK && il == 1 && t->uniform == 0) break;  // not a one-size batch
                    float best_ms = 1e30f;
                    for (int rep = 0; rep < 3 && rc == LBM_OK; ++rep) {  // the second replays a graph
                        if (cudaEventRecord(e0, t->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
                        if (rc == LBM_OK) rc = lbm_batch_step(t, steps_per_trial);
                        if (rc == LBM_OK && (cudaEventRecord(e1, t->stream) != cudaSuccess ||
                                             cudaEventSynchronize(e1) != cudaSuccess))
                            rc = LBM_ERR_CUDA;
                        float ms = 0.0f;
                        if (rc == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms)
                            best_ms = ms;
                    }
                    const float us = best_ms * 1000.0f / (float)steps_per_trial;
                    if (rc == LBM_OK && us < best.us_per_step) {
                        best.rows = rows;
                        best.prefetch = pf_c[k];
                        best.interleave = il;
                        best.us_per_step = us;
                    }
                }
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (t) lbm_batch_destroy(t);
        for (lbm_handle s : scratch) lbm_destroy(s);
        if (rc != LBM_OK) return batch_err(rc < 0 ? rc : LBM_ERR_CUDA, "lbm_batch_autotune: trial failed");
        std::lock_guard<std::mutex> lock(g_btune_mutex);
        g_btune_cache.push_back(best);
    }
    const int rc = lbm_batch_set_launch(b, best.rows, best.prefetch, best.interleave);
    if (rc != LBM_OK) return rc;
    if (rows_out) *rows_out = best.rows;
    if (prefetch_out) *prefetch_out = best.prefetch;
    if (interleave_out) *interleave_out = best.interleave;
    if (us_per_step_out) *us_per_step_out = cached ? 0.0f : best.us_per_step;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// lbm_step_static: one diagnostic sweep on caller-owned buffers, with no
// allocation.  Its reduction scratch (per-block partials, tickets, the FP64
// record) lives in the file-scope device array below instead of memory the
// library would otherwise allocate per handle.
// ---------------------------------------------------------------------------
namespace {

constexpr unsigned kStaticMaxBlocks = 65536;  // ceil(nx / 128) * ny
constexpr unsigned kStaticMaxWall = 65536;    // heated-wall partials: ceil(nx / 128) or ny
constexpr size_t kStaticFold = (kStaticMaxBlocks + 1023) / 1024;
constexpr size_t kStaticOffRec = 256;
constexpr size_t kStaticOffQ = kStaticOffRec + 256;
constexpr size_t kStaticOffD = kStaticOffQ + (size_t)kStaticMaxWall * 8;
constexpr size_t kStaticOffD2 = kStaticOffD + (size_t)kStaticMaxBlocks * 32;
constexpr size_t kStaticBytes = kStaticOffD2 + ((kStaticFold * 32 + 255) / 256) * 256;  // ~2.6 MB

// Held by every GPU that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mutex;
void *g_static_addr[256] = {};  // device address of g_static_scratch, per device ordinal

}  // namespace

extern "C" int lbm_step_static(const void *src, void *dst, int nx, int ny, int precision,
                               const lbm_params *p, long long step, void *cuda_stream, lbm_diag *out) {
    if (!src || !dst || src == dst || !p || step < 0)
        return set_err(nullptr, LBM_ERR_ARG, "lbm_step_static: NULL or aliased buffers, or step < 0");
    if (nx < 2 || ny < 2 || ny > 65535)
        return set_err(nullptr, LBM_ERR_ARG, "lbm_step_static: need 2 <= nx, 2 <= ny <= 65535");
    if (precision != LBM_FP32 && precision != LBM_FP64)
        return set_err(nullptr, LBM_ERR_ARG, "lbm_step_static: precision must be LBM_FP32 or LBM_FP64");
    lbm_s t;  // launch description only; owns nothing
    t.nx = nx;
    t.ny = ny;
    t.precision = precision;
    t.ntx = (nx + kTW - 1) / kTW;
    t.rows = 1;
    t.prefetch = kDefaultPrefetch;
    set_grid(&t);
    const unsigned long long nblk = (unsigned long long)t.grid.x * t.grid.y;
    const int nq = p->problem == LBM_CAVITY ? (int)t.grid.x : (int)t.grid.y;
    if (nblk > kStaticMaxBlocks || (unsigned)nq > kStaticMaxWall)
        return set_err(nullptr, LBM_ERR_ARG,
                       "lbm_step_static: lattice too large for the static scratch (ceil(nx/128)*ny = %llu "
                       "> %u blocks); use lbm_create / lbm_step",
                       nblk, kStaticMaxBlocks);
    lbm_derived d;
    int rc = derive(&t, p, &d);
    if (rc != LBM_OK) {
        std::snprintf(g_create_error, sizeof(g_create_error), "lbm_step_static: %.200s", t.err);
        return rc;
    }
    t.p = *p;
    t.d = d;
    if (p->problem == LBM_CAVITY && p->strip_width > 0.0) {
        t.lo2 = (int)std::ceil(2.0 * d.a);
        t.hi2 = (int)std::floor(2.0 * d.b);
        t.strip_on = 1;
    }
    t.nq = nq;

    // Set-up, once per device with that device current: the array's name is a
    // host-side stand-in, so the kernels get its device address instead.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256)
        return set_err(nullptr, LBM_ERR_CUDA, "lbm_step_static: cudaGetDevice failed: %s",
                       cudaGetErrorString(e));
    char *base;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr)
                return set_err(nullptr, LBM_ERR_CUDA, "lbm_step_static: cudaGetSymbolAddress failed: %s",
                               cudaGetErrorString(e));
            g_static_addr[dev] = ptr;
        }
        base = static_cast<char *>(g_static_addr[dev]);
    }
    t.counters = reinterpret_cast<unsigned *>(base);
    t.rec = reinterpret_cast<DevRecord *>(base + kStaticOffRec);
    t.qpart = reinterpret_cast<double *>(base + kStaticOffQ);
    t.dpart = reinterpret_cast<double *>(base + kStaticOffD);
    t.dpart2 = reinterpret_cast<double *>(base + kStaticOffD2);
    t.stream = static_cast<cudaStream_t>(cuda_stream);

    // The array keeps the previous call's contents: the tickets and the record
    // must start from zero, and the record's step counter from `step`.
    const unsigned long long counter = (unsigned long long)step;
    e = cudaMemsetAsync(base, 0, kStaticOffQ, t.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&t.rec->counter, &counter, sizeof(counter), cudaMemcpyHostToDevice, t.stream);
    if (e != cudaSuccess)
        return set_err(nullptr, LBM_ERR_CUDA, "lbm_step_static: clearing the scratch failed: %s",
                       cudaGetErrorString(e));
    t.step = step;
    if (precision == LBM_FP64) {
        SweepArgs<double> a = make_args<double>(&t, src, dst);
        a.step = step + 1;
        e = launch_lattice<double, double>(a, p->problem, p->flow_on != 0, kSweepDiag, t.grid, t.block,
                                           t.stream, false);
    } else {
        SweepArgs<float> a = make_args<float>(&t, src, dst);
        a.step = step + 1;
        e = launch_lattice<float, float>(a, p->problem, p->flow_on != 0, kSweepDiag, t.grid, t.block,
                                         t.stream, false);
    }
    if (e != cudaSuccess)
        return set_err(nullptr, LBM_ERR_CUDA, "lbm_step_static: launch failed: %s", cudaGetErrorString(e));
    if (!out) return LBM_OK;
    DevRecord r;
    e = cudaMemcpyAsync(&r, t.rec, sizeof(r), cudaMemcpyDeviceToHost, t.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t.stream);
    if (e != cudaSuccess)
        return set_err(nullptr, LBM_ERR_CUDA, "lbm_step_static: reading the record failed: %s",
                       cudaGetErrorString(e));
    const double P = (double)nx * (double)ny;
    out->step = step + 1;
    out->melt_fraction = r.melt_sum / P;
    out->H_total = r.H_sum;
    out->Q_strip = r.Q_last;
    out->Q_cum = r.Q_cum;
    out->Nu = d.heated_len > 0.0 ? r.Q_last * d.Href / (d.alpha * d.heated_len) : 0.0;
    out->front_x = r.melt_sum / (double)ny;
    out->max_u = r.max_u;
    out->nan_flag = r.nan_flag != 0.0 ? 1 : 0;
    if (out->nan_flag) return set_err(nullptr, LBM_ERR_DIVERGED, "lbm_step_static: non-finite H or rho");
    return LBM_OK;
}
