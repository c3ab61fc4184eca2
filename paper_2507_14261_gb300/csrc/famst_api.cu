// C ABI of the FAMST library (include/famst.h): context, workspace,
// argument and device-side validation, and the phase and build entry
// points that string the kernels together in the order of Algorithm 1.
#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "batch.cuh"

#include "famst_internal.cuh"

using namespace famst;

// The last batched build's plan and its instantiated CUDA graph.
struct BatchCache {
    bool valid = false;
    std::vector<int64_t> offsets;
    std::vector<int32_t> dims;
    int B = 0, k = 0, lambda = 0, prec = 0, max_iters = 0;
    uint64_t seed = 0;
    const float *X = nullptr;
    int32_t *tu = nullptr, *tv = nullptr;
    float *tw = nullptr;
    BatchPlan plan;
    BatchHost host;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long graph_kernels = 0;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        if (host.W) cudaFreeHost(host.W);
        if (host.cbase) cudaFreeHost(host.cbase);
        if (host.hist) cudaFreeHost(host.hist);
        if (host.words) cudaFreeHost(host.words);
        host = BatchHost();
        valid = false;
    }
};

struct famst_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 1;
    unsigned long long launches = 0;
    // workspace slots: 0 = Phase 1 outputs and scratch, 1 = later phases,
    // 2 = device copies made by famst_build_host, 3 = batched builds
    char *ws[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t ws_cap[4] = {0, 0, 0, 0};
    cudaStream_t bstream = nullptr;  // private stream of batched builds (graph capture)
    // second stream of a build: the refinement's lists are built on it while
    // Algorithm 3 runs on the build's stream (fork / join events)
    cudaStream_t astream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    BatchCache batch;
    int *dstatus = nullptr;       // device status word
    int32_t *pinned = nullptr;    // 128 bytes of pinned host memory, slots PIN_*
    double *dW = nullptr;         // device: W, W64
    int prune = 1;                // Phase 1 tile pruning
    int loop_limit = 0;           // bounded loops: 0 = defaults (famst_set_loop_limit)
    int connect_mode = FAMST_CONNECT_RANDOM;
    // Phase 1 of builds: exact tiles or NN-Descent (famst_set_knn_method)
    int knn_method = FAMST_KNN_EXACT, nnd_S = 0, nnd_iters = 10;
    double nnd_delta = 0.001;
    int32_t knn_iters = 0;        // NN-Descent iterations of the last build
    KernelTimers timers;          // per-kernel events of a build with info
    bool timers_made = false, timing = false;
    double tile_fraction = 1.0;   // of the last Phase 1
    char err[256] = {0};
};

namespace {

// slots of the pinned host words: status word, component count, MST counter
constexpr int PIN_STATUS = 0, PIN_T = 4, PIN_MST = 8, PIN_KNN = 12, PIN_REF = 14, PIN_NND = 16;

// Record the first error of a call (the innermost, most specific one).
famst_status fail(famst_ctx *c, famst_status s, const char *msg) {
    if (!c || c->err[0]) return s;
    if (s == FAMST_ERR_CUDA)
        snprintf(c->err, sizeof(c->err), "%s: %s", msg, cudaGetErrorString(cudaGetLastError()));
    else
        snprintf(c->err, sizeof(c->err), "%s", msg);
    return s;
}

famst_status cuda_fail(famst_ctx *c, cudaError_t e, const char *where) {
    if (c && !c->err[0]) snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
    return FAMST_ERR_CUDA;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

#define ST(call)                                                   \
    do {                                                           \
        famst_status s_ = (call);                                  \
        if (s_ != FAMST_OK) return fail(ctx, s_, #call);           \
    } while (0)

// Make workspace slot `slot` hold at least `bytes`; returns an arena.
famst_status ensure_ws(famst_ctx *ctx, int slot, size_t bytes, Arena &ar) {
    bytes = align256(bytes) + 4096;
    if (bytes > ctx->ws_cap[slot]) {
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->ws[slot]) cudaFree(ctx->ws[slot]);
        ctx->ws[slot] = nullptr;
        ctx->ws_cap[slot] = 0;
        size_t want = bytes + bytes / 4;
        if (cudaMalloc(&ctx->ws[slot], want) != cudaSuccess) {
            cudaGetLastError();
            if (cudaMalloc(&ctx->ws[slot], bytes) != cudaSuccess) {
                cudaGetLastError();
                ctx->ws[slot] = nullptr;
                return fail(ctx, FAMST_ERR_OOM, "workspace allocation failed");
            }
            want = bytes;
        }
        ctx->ws_cap[slot] = want;
    }
    ar.base = ctx->ws[slot];
    ar.cap = ctx->ws_cap[slot];
    ar.off = 0;
    return FAMST_OK;
}

Exec exec_of(famst_ctx *ctx) {
    Exec e{ctx->stream, &ctx->launches, ctx->num_sms, ctx->dstatus};
    e.loop_limit = ctx->loop_limit;
    e.timers = ctx->timing ? &ctx->timers : nullptr;
    return e;
}

// Per-kernel timers for one build (created on first use, kept by the context).
struct TimingScope {
    famst_ctx *ctx;
    TimingScope(famst_ctx *c, bool on) : ctx(c) {
        if (!on) return;
        if (!ctx->timers_made) {
            for (auto &e : ctx->timers.ev)
                if (cudaEventCreate(&e) != cudaSuccess) return;
            ctx->timers_made = true;
        }
        for (auto &u : ctx->timers.used) u = false;
        ctx->timing = true;
    }
    double ms(int slot) const {
        float f = 0.0f;
        if (!ctx->timing || !ctx->timers.used[slot]) return 0.0;
        if (cudaEventElapsedTime(&f, ctx->timers.ev[2 * slot], ctx->timers.ev[2 * slot + 1]) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0.0;
        }
        return double(f);
    }
    ~TimingScope() { ctx->timing = false; }
};

__global__ void check_finite_kernel(const float *__restrict__ X, int64_t count, int *dstatus) {
    int bad = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        bad |= !isfinite(X[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(dstatus, STATUS_NONFINITE);
}


// ids in [0, n); for the kNN lists also != own row
__global__ void check_ids_kernel(const int32_t *__restrict__ ids, int64_t count, int64_t n, int k,
                                 int *dstatus) {
    int bad = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x) {
        int v = ids[i];
        bad |= (v < 0) | (int64_t(v) >= n);
        if (k > 0) bad |= (int64_t(v) == i / k);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(dstatus, STATUS_BAD_ID);
}

__global__ void check_off_kernel(const int32_t *__restrict__ off, int64_t t, int *dstatus) {
    int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c < t && off[c] < 0) set_status(dstatus, STATUS_BAD_ID);
}

// inter-component edges: ends in range and in the components they claim
__global__ void check_edges_kernel(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                                   const int32_t *__restrict__ eci,
                                   const int32_t *__restrict__ ecj,
                                   const int32_t *__restrict__ comp, int64_t m, int64_t n,
                                   int *dstatus) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    int u = eu[e], v = ev[e];
    bool bad = u < 0 || v < 0 || int64_t(u) >= n || int64_t(v) >= n;
    if (!bad && comp) bad = comp[u] != eci[e] || comp[v] != ecj[e] || eci[e] == ecj[e];
    if (bad) set_status(dstatus, STATUS_BAD_ID);
}

__global__ void max_i32_kernel(const int32_t *__restrict__ a, int64_t count, int32_t *out) {
    int mx = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        mx = a[i] > mx ? a[i] : mx;
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

unsigned grid_cap(famst_ctx *ctx, int64_t count, int th) {
    int64_t g = (count + th - 1) / th;
    int64_t cap = int64_t(ctx->num_sms) * 8;
    if (g > cap) g = cap;
    return unsigned(g < 1 ? 1 : g);
}

famst_status reset_status(famst_ctx *ctx) {
    CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), ctx->stream));
    return FAMST_OK;
}

// Synchronise and translate the device status word.
famst_status sync_status(famst_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->pinned + PIN_STATUS, ctx->dstatus, sizeof(int),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    int s = ctx->pinned[PIN_STATUS];
    if (s & STATUS_NONFINITE) return fail(ctx, FAMST_ERR_NONFINITE, "X holds NaN or Inf");
    if (s & STATUS_BAD_ID) return fail(ctx, FAMST_ERR_INVALID_ARG, "vertex id out of range or inconsistent");
    if (s & STATUS_LOOP_LIMIT) return fail(ctx, FAMST_ERR_TIMEOUT, "a bounded device loop reached its limit");
    if (s & STATUS_REFINE_CAP) return fail(ctx, FAMST_ERR_NO_CONVERGENCE, "refinement reached max_iters");
    if (s & STATUS_DISCONNECTED) return fail(ctx, FAMST_ERR_DISCONNECTED, "graph is not connected");
    if (s & STATUS_INTERNAL) return fail(ctx, FAMST_ERR_CUDA, "internal buffer bound exceeded");
    return FAMST_OK;
}

bool vec4_ok(const float *X, int d) {
    return (d % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
}

famst_status check_points(famst_ctx *ctx, const float *X, int64_t n, int32_t d) {
    if (!X) return fail(ctx, FAMST_ERR_INVALID_ARG, "X is NULL");
    if (n < 1 || d < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "need n >= 1 and d >= 1");
    if (n >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "n must be < 2^31");
    Exec ex = exec_of(ctx);
    FAMST_LAUNCH(ex, check_finite_kernel, grid_cap(ctx, n * d, 256), 256, 0, X, n * d,
                 ctx->dstatus);
    return FAMST_OK;
}

famst_status check_knn_args(famst_ctx *ctx, int64_t n, int32_t k) {
    if (k < 1 || int64_t(k) > n - 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= k <= n-1");
    if (k > 128) return fail(ctx, FAMST_ERR_UNSUPPORTED, "k > 128");
    if (n * int64_t(k) >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "n*k must be < 2^31");
    return FAMST_OK;
}

famst_status check_nbr(famst_ctx *ctx, const int32_t *nbr, int64_t n, int32_t k) {
    if (!nbr) return fail(ctx, FAMST_ERR_INVALID_ARG, "nbr is NULL");
    Exec ex = exec_of(ctx);
    FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, n * k, 256), 256, 0, nbr, n * k, n, k,
                 ctx->dstatus);
    return FAMST_OK;
}

// ---------------------------------------------------------- stage helpers

// Debug build (compiled with FAMST_CHECK_BOUNDS: libfamst_checked.so): every
// index array that one build stage hands to the next is validated on the
// device before the next stage gathers with it -- kNN ids in [0, n) and not
// the row itself, component labels in [0, t), member lists and offsets,
// inter-component edges in range and in the components they claim (after
// Alg. 3 and after Alg. 4), tree edges in range. A violation fails the call
// with FAMST_ERR_CUDA and names the stage; nothing traps. Release builds
// compile all of this away.
#ifdef FAMST_CHECK_BOUNDS
famst_status debug_check(famst_ctx *ctx, const char *after) {
    CK(cudaMemcpyAsync(ctx->pinned + PIN_STATUS, ctx->dstatus, sizeof(int),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->pinned[PIN_STATUS] & STATUS_BAD_ID) {
        snprintf(ctx->err, sizeof(ctx->err), "bounds check failed after %s", after);
        return FAMST_ERR_CUDA;
    }
    return FAMST_OK;
}
#define FAMST_DEBUG_IDS(ids, count, range, k, after)                                            \
    do {                                                                                      \
        FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, (count), 256), 256, 0, (ids),        \
                     int64_t(count), int64_t(range), (k), ctx->dstatus);                      \
        ST(debug_check(ctx, after));                                                          \
    } while (0)
#define FAMST_DEBUG_EDGES(after)                                                              \
    do {                                                                                      \
        if (m > 0)                                                                            \
            FAMST_LAUNCH(ex, check_edges_kernel, unsigned((m + 255) / 256), 256, 0, eu, evv,  \
                         eci, ecj, comp, m, n, ctx->dstatus);                                 \
        ST(debug_check(ctx, after));                                                          \
    } while (0)
#else
#define FAMST_DEBUG_IDS(ids, count, range, k, after) do { } while (0)
#define FAMST_DEBUG_EDGES(after) do { } while (0)
#endif

// Stage boundaries of a build: CUDA events (when statistics were asked
// for) and NVTX ranges on the host thread, one range per stage, so that a
// profiler can attribute kernels to the paper's phases (NVTX is header-only
// and costs nothing when no tool listens).
struct Events {
    cudaEvent_t e[8] = {};
    int used = 0;
    bool on = false;
    bool range_open = false;
    void init(bool enable) {
        on = enable;
        if (on)
            for (auto &x : e) cudaEventCreate(&x);
    }
    void mark(cudaStream_t s, int i) {
        static const char *const stage[5] = {
            "famst: Phase 1 kNN graph", "famst: Alg. 2 components", "famst: Alg. 3 connect",
            "famst: Alg. 4 refine", "famst: MST and tree weight"};
        if (on) cudaEventRecord(e[i], s);
        if (i + 1 > used) used = i + 1;
        if (range_open) nvtxRangePop();
        range_open = i < 5;
        if (range_open) nvtxRangePushA(stage[i]);
    }
    double ms(int a, int b) {
        float f = 0.0f;
        if (on) cudaEventElapsedTime(&f, e[a], e[b]);
        return double(f);
    }
    ~Events() {
        if (range_open) nvtxRangePop();
        if (on)
            for (auto &x : e) cudaEventDestroy(x);
    }
};

// Phase 1 dispatch. Tensor precisions use the tcgen05 tiles when the shape
// fits them (k <= 63, operand rows fit shared memory); otherwise the FP32
// tiles compute every row (reported as uncertified rows).
famst_status knn_stage(famst_ctx *ctx, Arena &ar, const float *X, int64_t n, int32_t d, int32_t k,
                       int32_t prec, int32_t *nbr, float *dist, int64_t *uncert) {
    Exec ex = exec_of(ctx);
    *uncert = 0;
    if (prec != FAMST_PREC_FP32) {
        const bool x3 = prec == FAMST_PREC_BF16X3, f8 = prec == FAMST_PREC_FP8;
        if (knn_tc_supported(n, d, k, x3, f8)) {
            int64_t visited = 0;
            ctx->tile_fraction = 1.0;
            famst_status st = knn_tc(ex, ar, X, n, d, k, x3, vec4_ok(X, d), nbr, dist,
                                     ctx->pinned + PIN_KNN, uncert, nullptr,
                                     ctx->prune != 0 && !f8, &visited, f8);
            const double all = double((n + 127) / 128) * double((n + 255) / 256);
            if (st == FAMST_OK) ctx->tile_fraction = double(visited) / all;
            return st;
        }
        *uncert = n;
    }
    return knn_fp32(ex, ar, X, n, d, k, nullptr, 0, n, nbr, dist);
}

size_t knn_stage_ws(famst_ctx *ctx, int64_t n, int32_t d, int32_t k, int32_t prec) {
    const bool f8 = prec == FAMST_PREC_FP8;
    if (prec != FAMST_PREC_FP32 && knn_tc_supported(n, d, k, prec == FAMST_PREC_BF16X3, f8))
        return knn_tc_workspace(n, d, k, prec == FAMST_PREC_BF16X3, ctx->num_sms,
                                !f8 && ctx->prune != 0 && prune_supported(n, d, k, true), f8);
    return knn_fp32_workspace(n, d, k, n, ctx->num_sms);
}

// Workspace of Phases 2-3 + MST (slot 1) for m inter-component edges.
size_t rest_ws(int64_t n, int32_t d, int32_t k, int64_t m, int64_t t, int32_t max_iters,
               int lambda_nearest = 0) {
    return (lambda_nearest > 0 ? connect_nearest_workspace(n, t, lambda_nearest) : 0) + align256(size_t(n) * 4) + align256(size_t(n + 1) * 4) + member_lists_workspace(n, t) +
           5 * align256(size_t(m > 0 ? m : 1) * 4) + align256(size_t(n + 1) * 4) +
           align256(size_t(n) * k * 4) + reverse_csr_workspace(n, k) +
           align256(size_t(max_iters + 1) * 4) + refine_workspace(m) +
           boruvka_workspace(n, n * int64_t(k) + m) + tree_weight_workspace(n) +
           half_rows_workspace(n, d) + glists_workspace(n, k) + refine_build_workspace(n, m) +
           4096;
}

// Workspace of Phase 1 inside a build (slot 0): nbr, dist, comp + the tiles.
size_t build_knn_ws(famst_ctx *ctx, int64_t n, int32_t d, int32_t k, int32_t prec) {
    return 2 * align256(size_t(n) * k * 4) + align256(size_t(n) * 4) +
           knn_stage_ws(ctx, n, d, k, prec) + 4096;
}

// Phases 2-3 + MST on device data. nbr/dist come from Phase 1.
struct BuildOut {
    int32_t *tu, *tv;
    float *tw;
};

famst_status build_rest(famst_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t k,
                        int32_t lambda, uint64_t seed, int32_t max_iters, const int32_t *nbr,
                        const float *dist, int32_t *comp, BuildOut out, double *W_out,
                        famst_build_info *info, Events &ev) {
    Exec ex = exec_of(ctx);
    const bool v4 = vec4_ok(X, d);
    Arena ar;
    // components
    ST(ensure_ws(ctx, 1, components_workspace(n) + 256, ar));
    int32_t *t_dev = ar.take<int32_t>(1);
    ST(components_uf(ex, ar, nbr, n, k, comp, t_dev));
    CK(cudaMemcpyAsync(ctx->pinned + PIN_T, t_dev, 4, cudaMemcpyDeviceToHost, ctx->stream));
    ST(sync_status(ctx));
    const int64_t t = ctx->pinned[PIN_T];
    FAMST_DEBUG_IDS(comp, n, t, 0, "Alg. 2 (component labels)");
    ev.mark(ctx->stream, 2);
    const int64_t m = int64_t(lambda) * t * (t - 1) / 2;
    if (m >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "lambda*t*(t-1)/2 >= 2^31");
    // workspace for connect, refine and MST
    ST(ensure_ws(ctx, 1,
                 rest_ws(n, d, k, m, t, max_iters,
                         ctx->connect_mode == FAMST_CONNECT_NEAREST ? lambda : 0),
                 ar));
    int32_t *members = ar.take<int32_t>(size_t(n));
    int32_t *comp_off = ar.take<int32_t>(size_t(n + 1));
    int32_t *eu = ar.take<int32_t>(size_t(m > 0 ? m : 1));
    int32_t *evv = ar.take<int32_t>(size_t(m > 0 ? m : 1));
    float *ew = ar.take<float>(size_t(m > 0 ? m : 1));
    int32_t *eci = ar.take<int32_t>(size_t(m > 0 ? m : 1));
    int32_t *ecj = ar.take<int32_t>(size_t(m > 0 ? m : 1));
    int32_t *hist = ar.take<int32_t>(size_t(max_iters + 1));
    unsigned long long *evals = ar.take<unsigned long long>(4);
    // the components kernels above used this slot; comp lives in slot 0
    int sweeps = 0, filter = -1;
    unsigned long long evals_host[4] = {0, 0, 0, 0};
    int64_t first_delta = 0;
    if (t > 1) {
        ST(member_lists(ex, ar, comp, n, t, members, comp_off));
        FAMST_DEBUG_IDS(members, n, n, 0, "member lists");
        FAMST_DEBUG_IDS(comp_off, t + 1, n + 1, 0, "member list offsets");
        // BF16 copies of the points for the Alg. 4 filter (half the bytes per
        // candidate; exactness comes from the canonical survivors) and for the
        // nearest-pair connect
        HalfRows hr;
        const bool nearest = ctx->connect_mode == FAMST_CONNECT_NEAREST;
        const bool use_half = v4 && d >= 32 && d <= 256;   // the refinement's BF16 filter
        if (use_half || nearest) ST(half_rows(ex, ar, X, n, d, &hr));
        int32_t *rev_off = ar.take<int32_t>(size_t(n + 1));
        int32_t *rev_src = ar.take<int32_t>(size_t(n) * k);
        if (!rev_off || !rev_src || !hist) return fail(ctx, FAMST_ERR_OOM, "workspace");
        // work left on the second stream is waited for if this call fails
        struct AuxGuard {
            cudaStream_t s = nullptr;
            ~AuxGuard() {
                if (s) cudaStreamSynchronize(s);
            }
        } aux;
        bool forked = false;
        if (nearest) {
            if (d > 256) return fail(ctx, FAMST_ERR_UNSUPPORTED, "the nearest-pair connect needs d <= 256");
            std::vector<int32_t> off_h(size_t(t + 1));
            CK(cudaMemcpyAsync(off_h.data(), comp_off, size_t(t + 1) * 4, cudaMemcpyDeviceToHost,
                               ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            const size_t mark = ar.off;   // the lists are scratch of this step
            ST(connect_nearest(ex, ar, X, d, hr, members, comp_off, off_h.data(), t, lambda, eu,
                               evv, ew, eci, ecj, nullptr));
            ar.off = mark;
        } else {
            if (use_half) {
                // the refinement's lists (reverse kNN lists, deduplicated G
                // lists) do not depend on Alg. 3: built on the second stream
                // while Alg. 3 runs (Alg. 3 allocates no workspace)
                CK(cudaEventRecord(ctx->fork_ev, ctx->stream));
                CK(cudaStreamWaitEvent(ctx->astream, ctx->fork_ev, 0));
                aux.s = ctx->astream;
                Exec ax = ex;
                ax.stream = ctx->astream;
                ax.timers = nullptr;
                ST(reverse_csr(ax, ar, nbr, n, k, rev_off, rev_src));
                ST(refine_glists(ax, ar, nbr, n, k, rev_off, rev_src, &hr));
                CK(cudaEventRecord(ctx->join_ev, ctx->astream));
                forked = true;
            }
            ST(connect_edges(ex, X, d, v4, members, comp_off, t, lambda, seed, eu, evv, ew, eci,
                             ecj, hr.h ? &hr : nullptr));
        }
        FAMST_DEBUG_EDGES("Alg. 3 (inter-component edges)");
        ev.mark(ctx->stream, 3);
        if (!use_half) hr = HalfRows();   // only the refinement filter uses them
        if (forked) {
            CK(cudaStreamWaitEvent(ctx->stream, ctx->join_ev, 0));
            aux.s = nullptr;   // later work on the build's stream is ordered after it
        } else {
            ST(reverse_csr(ex, ar, nbr, n, k, rev_off, rev_src));
            ST(refine_glists(ex, ar, nbr, n, k, rev_off, rev_src, &hr));
        }
        CK(cudaMemsetAsync(hist, 0, size_t(max_iters + 1) * 4, ctx->stream));
        if (!evals) return fail(ctx, FAMST_ERR_OOM, "workspace");
        CK(cudaMemsetAsync(evals, 0, 32, ctx->stream));
        if (refine_staged_supported(hr)) {   // BF16 rows staged in shared memory
            filter = REFINE_FILTER_BF16_MMA;
            ST(refine_build(ex, ar, X, d, hr, members, n, eu, evv, ew, nullptr, m, max_iters, hist,
                            evals, ctx->pinned + PIN_REF));
        } else {
            ST(refine_edges(ex, ar, X, d, v4, nbr, k, rev_off, rev_src, comp, t, eu, evv, ew, eci,
                            ecj, m, max_iters, hist, evals, false, &filter));
        }
        FAMST_DEBUG_EDGES("Alg. 4 (refined edges)");
        ev.mark(ctx->stream, 4);
        famst_status s = sync_status(ctx);
        if (s != FAMST_OK) return s;
        // sweeps = 1 + largest change count; |Delta_1| = edges that changed at least once
        int32_t *hh = new (std::nothrow) int32_t[max_iters + 1];
        if (!hh) return fail(ctx, FAMST_ERR_OOM, "host");
        CK(cudaMemcpy(hh, hist, size_t(max_iters + 1) * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(evals_host, evals, 32, cudaMemcpyDeviceToHost));
        for (int c = 0; c <= max_iters; ++c)
            if (hh[c]) sweeps = c + 1;
        first_delta = m - hh[0];
        delete[] hh;
    } else {
        ev.mark(ctx->stream, 3);
        ev.mark(ctx->stream, 4);
        sweeps = 0;
    }
    int64_t got = 0;
    int rounds = 0;
    // an NN-Descent graph is not the exact kNN: a vertex's lightest edge may
    // come from another vertex's list
    ST(boruvka(ex, ar, n, nbr, dist, k, eu, evv, ew, m, MstOut{out.tu, out.tv, out.tw}, &got,
               &rounds, ctx->pinned + PIN_MST, ctx->knn_method != FAMST_KNN_NNDESCENT, true));
    if (got != n - 1) return fail(ctx, FAMST_ERR_DISCONNECTED, "candidate graph is not connected");
    FAMST_DEBUG_IDS(out.tu, n - 1, n, 0, "MST (tree edge ends)");
    FAMST_DEBUG_IDS(out.tv, n - 1, n, 0, "MST (tree edge ends)");
    ST(tree_weight(ex, ar, X, d, v4, out.tu, out.tv, out.tw, n - 1, ctx->dW));
    ev.mark(ctx->stream, 5);
    double W[2];
    CK(cudaMemcpyAsync(W, ctx->dW, 16, cudaMemcpyDeviceToHost, ctx->stream));
    ST(sync_status(ctx));
    if (W_out) *W_out = W[0];
    if (info) {
        info->t = t;
        info->m = m;
        info->refine_sweeps = sweeps;
        info->boruvka_rounds = rounds;
        info->first_delta = first_delta;
        info->refine_distance_evals = int64_t(evals_host[0]);
        info->refine_canonical_evals = int64_t(evals_host[1]);
        info->refine_filter = filter;
        info->refine_rows_staged = int64_t(evals_host[2]);
        info->refine_fixed_rows = int64_t(evals_host[3]);
        info->W = W[0];
        info->W64 = W[1];
    }
    return FAMST_OK;
}

famst_status build_impl(famst_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t k,
                        int32_t lambda, uint64_t seed, int32_t prec, int32_t max_iters,
                        BuildOut out, double *W_out, famst_build_info *info) {
    if (lambda < 1 || lambda > 32) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= lambda <= 32");
    if (max_iters < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "need max_iters >= 1");
    if (prec < 0 || prec > 3) return fail(ctx, FAMST_ERR_INVALID_ARG, "unknown precision");
    if (info) memset(info, 0, sizeof(*info));
    if (n == 1) {
        if (W_out) *W_out = 0.0;
        return FAMST_OK;
    }
    ST(check_knn_args(ctx, n, k));
    Events ev;
    ev.init(info != nullptr);
    TimingScope tscope(ctx, info != nullptr);
    ev.mark(ctx->stream, 0);
    ST(reset_status(ctx));
    ST(check_points(ctx, X, n, d));
    ST(sync_status(ctx));
    Arena ar;
    const bool nnd = ctx->knn_method == FAMST_KNN_NNDESCENT;
    const int S = ctx->nnd_S > 0 ? ctx->nnd_S : (k < 32 ? k : 32);
    if (nnd && !nndescent_supported(n, d, k, S))
        return fail(ctx, FAMST_ERR_UNSUPPORTED, "NN-Descent needs k <= 32, S <= 32, 2 S d floats in shared memory");
    ST(ensure_ws(ctx, 0, nnd ? align256(size_t(n) * k * 8) + align256(size_t(n) * 4) +
                                   nndescent_workspace(n, d, k, S) + 4096
                             : build_knn_ws(ctx, n, d, k, prec), ar));
    int32_t *nbr = ar.take<int32_t>(size_t(n) * k);
    float *dist = ar.take<float>(size_t(n) * k);
    int32_t *comp = ar.take<int32_t>(size_t(n));
    int64_t uncert = 0;
    ctx->knn_iters = 0;
    if (nnd) {
        // the build's seed; the draws' counters (tags 1, 2) differ from Alg. 3's (0)
        const size_t mark = ar.off;
        ST(nndescent(exec_of(ctx), ar, X, n, d, k, S, ctx->nnd_iters, ctx->nnd_delta, seed,
                     nullptr, nbr, dist, ctx->pinned + PIN_NND, &ctx->knn_iters, nullptr,
                     nullptr));
        ar.off = mark;
    } else {
        ST(knn_stage(ctx, ar, X, n, d, k, prec, nbr, dist, &uncert));
    }
#ifdef FAMST_CHECK_BOUNDS
    {
        Exec ex = exec_of(ctx);
        FAMST_DEBUG_IDS(nbr, n * k, n, k, "Phase 1 (kNN ids)");
    }
#endif
    ev.mark(ctx->stream, 1);
    famst_status s = build_rest(ctx, X, n, d, k, lambda, seed, max_iters, nbr, dist, comp, out,
                                W_out, info, ev);
    if (s != FAMST_OK) return s;
    if (info) {
        CK(cudaStreamSynchronize(ctx->stream));
        info->uncertified_rows = uncert;
        info->knn_tile_fraction = prec == FAMST_PREC_FP32 || nnd ? 1.0 : ctx->tile_fraction;
        info->knn_iters = ctx->knn_iters;
        info->ms_knn = ev.ms(0, 1);
        info->ms_components = ev.ms(1, 2);
        info->ms_connect = ev.ms(2, 3);
        info->ms_refine = ev.ms(3, 4);
        info->ms_mst = ev.ms(4, 5);
        info->ms_total = ev.ms(0, 5);
        info->ms_knn_tiles = tscope.ms(TIMER_TILES);
        info->ms_rerank = tscope.ms(TIMER_RERANK);
        info->ms_connect_kernel = tscope.ms(TIMER_CONNECT);
        info->ms_refine_kernel = tscope.ms(TIMER_REFINE);
    }
    return FAMST_OK;
}

}  // namespace

// ================================================================== C ABI

extern "C" {

famst_status famst_create(famst_ctx **out, int device) {
    if (!out) return FAMST_ERR_INVALID_ARG;
    *out = nullptr;
    famst_ctx *ctx = new (std::nothrow) famst_ctx();
    if (!ctx) return FAMST_ERR_OOM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dstatus, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dW, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->pinned, 128);
    if (e == cudaSuccess) e = cudaMemset(ctx->dstatus, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->astream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        famst_destroy(ctx);
        return FAMST_ERR_CUDA;
    }
    *out = ctx;
    return FAMST_OK;
}

famst_status famst_destroy(famst_ctx *ctx) {
    if (!ctx) return FAMST_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->batch.release();
    if (ctx->bstream) cudaStreamDestroy(ctx->bstream);
    if (ctx->astream) {
        cudaStreamSynchronize(ctx->astream);
        cudaStreamDestroy(ctx->astream);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    for (int i = 0; i < 4; ++i)
        if (ctx->ws[i]) cudaFree(ctx->ws[i]);
    if (ctx->dstatus) cudaFree(ctx->dstatus);
    if (ctx->dW) cudaFree(ctx->dW);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->timers_made)
        for (auto &e : ctx->timers.ev) cudaEventDestroy(e);
    delete ctx;
    return FAMST_OK;
}

famst_status famst_set_stream(famst_ctx *ctx, void *stream) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return FAMST_OK;
}

famst_status famst_workspace_query(famst_ctx *ctx, int64_t n, int32_t d, int32_t k,
                                   int32_t lambda, int64_t t_max, int32_t prec,
                                   int32_t max_iters, size_t *bytes) {
    if (!ctx || !bytes) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    *bytes = 0;
    if (n < 1 || d < 1 || lambda < 1 || lambda > 32 || max_iters < 1 || prec < 0 || prec > 3 ||
        t_max < 1 || t_max > n)
        return fail(ctx, FAMST_ERR_INVALID_ARG, "bad shape");
    if (n == 1) return FAMST_OK;
    ST(check_knn_args(ctx, n, k));
    const int64_t m = int64_t(lambda) * t_max * (t_max - 1) / 2;
    if (m >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "lambda*t*(t-1)/2 >= 2^31");
    // as ensure_ws rounds a slot: aligned, plus its 4 KB guard
    *bytes = (align256(build_knn_ws(ctx, n, d, k, prec)) + 4096) +
             (align256(rest_ws(n, d, k, m, t_max, max_iters,
                               ctx->connect_mode == FAMST_CONNECT_NEAREST ? lambda : 0)) +
              4096);
    return FAMST_OK;
}

famst_status famst_set_connect_mode(famst_ctx *ctx, int32_t mode) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (mode != FAMST_CONNECT_RANDOM && mode != FAMST_CONNECT_NEAREST)
        return fail(ctx, FAMST_ERR_INVALID_ARG, "unknown connect mode");
    ctx->connect_mode = mode;
    return FAMST_OK;
}

famst_status famst_set_loop_limit(famst_ctx *ctx, int32_t limit) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (limit < 0) return fail(ctx, FAMST_ERR_INVALID_ARG, "need limit >= 0");
    ctx->loop_limit = limit;
    return FAMST_OK;
}

famst_status famst_set_knn_pruning(famst_ctx *ctx, int32_t enable) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    ctx->prune = enable ? 1 : 0;
    return FAMST_OK;
}

const char *famst_error_string(famst_status s) {
    switch (s) {
        case FAMST_OK: return "ok";
        case FAMST_ERR_INVALID_ARG: return "invalid argument";
        case FAMST_ERR_CAPACITY: return "output capacity too small";
        case FAMST_ERR_NO_CONVERGENCE: return "refinement did not converge within max_iters";
        case FAMST_ERR_TIMEOUT: return "bounded device loop gave up";
        case FAMST_ERR_CUDA: return "CUDA error";
        case FAMST_ERR_OOM: return "out of device memory";
        case FAMST_ERR_UNSUPPORTED: return "unsupported size or mode";
        case FAMST_ERR_NONFINITE: return "input holds NaN or Inf";
        case FAMST_ERR_DISCONNECTED: return "graph is not connected";
        default: return "unknown status";
    }
}

const char *famst_last_error(const famst_ctx *ctx) { return ctx ? ctx->err : ""; }

uint64_t famst_launch_count(const famst_ctx *ctx) { return ctx ? ctx->launches : 0; }

size_t famst_workspace_bytes(const famst_ctx *ctx) {
    return ctx ? ctx->ws_cap[0] + ctx->ws_cap[1] + ctx->ws_cap[2] + ctx->ws_cap[3] : 0;
}

famst_status famst_knn_graph(famst_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t k,
                             int32_t prec, int32_t *nbr, float *dist) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!nbr || !dist) return fail(ctx, FAMST_ERR_INVALID_ARG, "nbr/dist NULL");
    if (prec < 0 || prec > 3) return fail(ctx, FAMST_ERR_INVALID_ARG, "unknown precision");
    if (n < 2) return fail(ctx, FAMST_ERR_INVALID_ARG, "need n >= 2");
    ST(check_knn_args(ctx, n, k));
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_points(ctx, X, n, d));
    ST(sync_status(ctx));
    Arena ar;
    ST(ensure_ws(ctx, 0, knn_stage_ws(ctx, n, d, k, prec), ar));
    int64_t uncert = 0;
    ST(knn_stage(ctx, ar, X, n, d, k, prec, nbr, dist, &uncert));
    return sync_status(ctx);
}

famst_status famst_knn_nndescent(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                                 int32_t k, int32_t S, int32_t max_iters, double delta,
                                 uint64_t seed, const int32_t *init_nbr, int32_t *nbr,
                                 float *dist, int32_t *iters_out, int64_t *updates,
                                 int64_t *pairs) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!nbr || !dist) return fail(ctx, FAMST_ERR_INVALID_ARG, "nbr/dist NULL");
    if (n < 2) return fail(ctx, FAMST_ERR_INVALID_ARG, "need n >= 2");
    if (max_iters < 0 || !(delta >= 0.0)) return fail(ctx, FAMST_ERR_INVALID_ARG, "need max_iters >= 0, delta >= 0");
    if (S < 1 || S > 32) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= S <= 32");
    ST(check_knn_args(ctx, n, k));
    if (!nndescent_supported(n, d, k, S))
        return fail(ctx, FAMST_ERR_UNSUPPORTED, "NN-Descent needs k <= 32 and 2 S d floats in shared memory");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_points(ctx, X, n, d));
    ST(sync_status(ctx));
    Arena ar;
    ST(ensure_ws(ctx, 0, nndescent_workspace(n, d, k, S), ar));
    int32_t it = 0;
    ST(nndescent(exec_of(ctx), ar, X, n, d, k, S, max_iters, delta, seed, init_nbr, nbr, dist,
                 ctx->pinned + PIN_NND, &it, updates, pairs));
    if (iters_out) *iters_out = it;
    return sync_status(ctx);
}

famst_status famst_set_knn_method(famst_ctx *ctx, int32_t method, int32_t S, int32_t max_iters,
                                  double delta) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (method != FAMST_KNN_EXACT && method != FAMST_KNN_NNDESCENT)
        return fail(ctx, FAMST_ERR_INVALID_ARG, "unknown kNN method");
    if (S < 0 || S > 32 || max_iters < 0 || !(delta >= 0.0))
        return fail(ctx, FAMST_ERR_INVALID_ARG, "need 0 <= S <= 32, max_iters >= 0, delta >= 0");
    ctx->knn_method = method;
    ctx->nnd_S = S;
    ctx->nnd_iters = max_iters;
    ctx->nnd_delta = delta;
    return FAMST_OK;
}

famst_status famst_components(famst_ctx *ctx, const int32_t *nbr, int64_t n, int32_t k,
                              int32_t *comp, int64_t *t_out) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!comp || !t_out) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL output");
    if (n < 2) return fail(ctx, FAMST_ERR_INVALID_ARG, "need n >= 2");
    ST(check_knn_args(ctx, n, k));
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_nbr(ctx, nbr, n, k));
    ST(sync_status(ctx));
    Arena ar;
    ST(ensure_ws(ctx, 0, components_workspace(n) + 256, ar));
    int32_t *t_dev = ar.take<int32_t>(1);
    ST(components_uf(exec_of(ctx), ar, nbr, n, k, comp, t_dev));
    CK(cudaMemcpyAsync(ctx->pinned + PIN_T, t_dev, 4, cudaMemcpyDeviceToHost, ctx->stream));
    ST(sync_status(ctx));
    *t_out = ctx->pinned[PIN_T];
    return FAMST_OK;
}

famst_status famst_connect(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                           const int32_t *comp, int64_t t, int32_t lambda, uint64_t seed,
                           int32_t *eu, int32_t *ev, float *ew, int32_t *eci, int32_t *ecj,
                           int64_t capacity, int64_t *m_out) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!comp || !m_out) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL argument");
    if (lambda < 1 || lambda > 32) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= lambda <= 32");
    if (t < 1 || t > n) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= t <= n");
    const int64_t m = int64_t(lambda) * t * (t - 1) / 2;
    *m_out = m;
    if (m >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "lambda*t*(t-1)/2 >= 2^31");
    if (capacity < m) return fail(ctx, FAMST_ERR_CAPACITY, "edge arrays shorter than lambda*t*(t-1)/2");
    if (m > 0 && (!eu || !ev || !ew || !eci || !ecj)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL edge array");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_points(ctx, X, n, d));
    Exec ex = exec_of(ctx);
    FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, n, 256), 256, 0, comp, n, t, 0, ctx->dstatus);
    ST(sync_status(ctx));
    if (m == 0) return FAMST_OK;
    Arena ar;
    ST(ensure_ws(ctx, 1, align256(size_t(n) * 4) + align256(size_t(n + 1) * 4) +
                             member_lists_workspace(n, t), ar));
    int32_t *members = ar.take<int32_t>(size_t(n));
    int32_t *comp_off = ar.take<int32_t>(size_t(n + 1));
    CK(cudaMemsetAsync(comp_off, 0xff, size_t(n + 1) * 4, ctx->stream));
    ST(member_lists(ex, ar, comp, n, t, members, comp_off));
    FAMST_LAUNCH(ex, check_off_kernel, unsigned((t + 255) / 256), 256, 0, comp_off, t, ctx->dstatus);
    ST(sync_status(ctx));
    ST(connect_edges(ex, X, d, vec4_ok(X, d), members, comp_off, t, lambda, seed, eu, ev, ew, eci,
                     ecj));
    return sync_status(ctx);
}

famst_status famst_connect_nearest(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                                   const int32_t *comp, int64_t t, int32_t lambda,
                                   int32_t *eu, int32_t *ev, float *ew, int32_t *eci,
                                   int32_t *ecj, int64_t capacity, int64_t *m_out) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!comp || !m_out) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL argument");
    if (lambda < 1 || lambda > 32) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= lambda <= 32");
    if (t < 1 || t > n) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= t <= n");
    if (d > 256) return fail(ctx, FAMST_ERR_UNSUPPORTED, "the nearest-pair connect needs d <= 256");
    const int64_t m = int64_t(lambda) * t * (t - 1) / 2;
    *m_out = m;
    if (m >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "lambda*t*(t-1)/2 >= 2^31");
    if (capacity < m) return fail(ctx, FAMST_ERR_CAPACITY, "edge arrays shorter than lambda*t*(t-1)/2");
    if (m > 0 && (!eu || !ev || !ew || !eci || !ecj)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL edge array");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_points(ctx, X, n, d));
    Exec ex = exec_of(ctx);
    FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, n, 256), 256, 0, comp, n, t, 0, ctx->dstatus);
    ST(sync_status(ctx));
    if (m == 0) return FAMST_OK;
    Arena ar;
    ST(ensure_ws(ctx, 1, align256(size_t(n) * 4) + align256(size_t(n + 1) * 4) +
                             member_lists_workspace(n, t) + half_rows_workspace(n, d) +
                             connect_nearest_workspace(n, t, lambda), ar));
    int32_t *members = ar.take<int32_t>(size_t(n));
    int32_t *comp_off = ar.take<int32_t>(size_t(n + 1));
    CK(cudaMemsetAsync(comp_off, 0xff, size_t(n + 1) * 4, ctx->stream));
    ST(member_lists(ex, ar, comp, n, t, members, comp_off));
    FAMST_LAUNCH(ex, check_off_kernel, unsigned((t + 255) / 256), 256, 0, comp_off, t, ctx->dstatus);
    ST(sync_status(ctx));
    std::vector<int32_t> off_h(size_t(t + 1));
    CK(cudaMemcpy(off_h.data(), comp_off, size_t(t + 1) * 4, cudaMemcpyDeviceToHost));
    HalfRows hr;
    ST(half_rows(ex, ar, X, n, d, &hr));
    ST(connect_nearest(ex, ar, X, d, hr, members, comp_off, off_h.data(), t, lambda, eu, ev, ew,
                       eci, ecj, nullptr));
    return sync_status(ctx);
}

famst_status famst_refine(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                          const int32_t *nbr, int32_t k, const int32_t *comp, int32_t *eu,
                          int32_t *ev, float *ew, const int32_t *eci, const int32_t *ecj,
                          int64_t m, int32_t max_iters, int32_t *sweeps_out, int64_t *delta_hist) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!comp || !sweeps_out) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL argument");
    if (max_iters < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "need max_iters >= 1");
    if (m < 0) return fail(ctx, FAMST_ERR_INVALID_ARG, "m < 0");
    if (n < 2) return fail(ctx, FAMST_ERR_INVALID_ARG, "need n >= 2");
    ST(check_knn_args(ctx, n, k));
    if (m > 0 && (!eu || !ev || !ew || !eci || !ecj)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL edge array");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_points(ctx, X, n, d));
    ST(check_nbr(ctx, nbr, n, k));
    Exec ex = exec_of(ctx);
    FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, n, 256), 256, 0, comp, n, n, 0, ctx->dstatus);
    ST(sync_status(ctx));
    if (m > 0) {
        FAMST_LAUNCH(ex, check_edges_kernel, unsigned((m + 255) / 256), 256, 0, eu, ev, eci, ecj,
                     comp, m, n, ctx->dstatus);
        ST(sync_status(ctx));
    }
    *sweeps_out = 0;
    if (m == 0) {
        *sweeps_out = 1;
        if (delta_hist) delta_hist[0] = 0;
        return FAMST_OK;
    }
    Arena ar;
    ST(ensure_ws(ctx, 1, align256(size_t(n + 1) * 4) + align256(size_t(n) * k * 4) +
                             reverse_csr_workspace(n, k) + align256(size_t(max_iters + 1) * 4) +
                             refine_workspace(m) + 256,
                 ar));
    int32_t *rev_off = ar.take<int32_t>(size_t(n + 1));
    int32_t *rev_src = ar.take<int32_t>(size_t(n) * k);
    int32_t *hist = ar.take<int32_t>(size_t(max_iters + 1));
    ST(reverse_csr(ex, ar, nbr, n, k, rev_off, rev_src));
    CK(cudaMemsetAsync(hist, 0, size_t(max_iters + 1) * 4, ctx->stream));
    // number of components: one more than the largest component index in E
    int32_t *tmax = ar.take<int32_t>(1);
    CK(cudaMemsetAsync(tmax, 0, 4, ctx->stream));
    FAMST_LAUNCH(ex, max_i32_kernel, grid_cap(ctx, m, 256), 256, 0, ecj, m, tmax);
    CK(cudaMemcpyAsync(ctx->pinned + PIN_T, tmax, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t t_e = int64_t(ctx->pinned[PIN_T]) + 1;
    ST(refine_edges(ex, ar, X, d, vec4_ok(X, d), nbr, k, rev_off, rev_src, comp, t_e, eu, ev, ew, eci, ecj,
                    m, max_iters, hist));
    famst_status s = sync_status(ctx);
    int32_t *hh = new (std::nothrow) int32_t[max_iters + 1];
    if (!hh) return fail(ctx, FAMST_ERR_OOM, "host");
    cudaError_t e = cudaMemcpy(hh, hist, size_t(max_iters + 1) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete[] hh;
        return cuda_fail(ctx, e, "copy histogram");
    }
    int sweeps = 0;
    for (int c = 0; c <= max_iters; ++c)
        if (hh[c]) sweeps = c + 1;
    if (sweeps > max_iters) sweeps = max_iters;
    *sweeps_out = sweeps;
    if (delta_hist) {
        // |Delta| of sweep s = edges whose change count is >= s
        int64_t ge = 0;
        for (int sidx = max_iters; sidx >= 1; --sidx) {
            ge += hh[sidx];
            if (sidx - 1 < max_iters) delta_hist[sidx - 1] = ge;
        }
    }
    delete[] hh;
    return s;
}

famst_status famst_mst(famst_ctx *ctx, int64_t n, const int32_t *nbr, const float *dist,
                       int32_t k, const int32_t *eu, const int32_t *ev, const float *ew, int64_t m,
                       int32_t *tu, int32_t *tv, float *tw, double *W_out) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!W_out) return fail(ctx, FAMST_ERR_INVALID_ARG, "W_out NULL");
    if (n < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "need n >= 1");
    if (m < 0) return fail(ctx, FAMST_ERR_INVALID_ARG, "m < 0");
    *W_out = 0.0;
    if (n == 1) return FAMST_OK;
    if (!tu || !tv || !tw || !dist) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL argument");
    ST(check_knn_args(ctx, n, k));
    if (m > 0 && (!eu || !ev || !ew)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL edge array");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_nbr(ctx, nbr, n, k));
    Exec ex = exec_of(ctx);
    if (m > 0)
        FAMST_LAUNCH(ex, check_edges_kernel, unsigned((m + 255) / 256), 256, 0, eu, ev, nullptr,
                     nullptr, nullptr, m, n, ctx->dstatus);
    ST(sync_status(ctx));
    Arena ar;
    ST(ensure_ws(ctx, 1, boruvka_workspace(n) + tree_weight_workspace(n), ar));
    int64_t got = 0;
    int rounds = 0;
    ST(boruvka(ex, ar, n, nbr, dist, k, eu, ev, ew, m, MstOut{tu, tv, tw}, &got, &rounds,
               ctx->pinned + PIN_MST));
    ST(sync_status(ctx));
    if (got != n - 1) return fail(ctx, FAMST_ERR_DISCONNECTED, "candidate graph is not connected");
    ST(tree_weight(ex, ar, nullptr, 0, false, tu, tv, tw, n - 1, ctx->dW));
    double W[2];
    CK(cudaMemcpyAsync(W, ctx->dW, 16, cudaMemcpyDeviceToHost, ctx->stream));
    ST(sync_status(ctx));
    *W_out = W[0];
    return FAMST_OK;
}

famst_status famst_emst_exact(famst_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t prec,
                              int32_t *tu, int32_t *tv, float *tw, double *W_out,
                              int32_t *rounds_out) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!W_out) return fail(ctx, FAMST_ERR_INVALID_ARG, "W_out NULL");
    if (prec == FAMST_PREC_FP8) return fail(ctx, FAMST_ERR_UNSUPPORTED, "FP8 tiles: kNN graph and build only");
    if (prec < 0 || prec > 2) return fail(ctx, FAMST_ERR_INVALID_ARG, "unknown precision");
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= n < 2^31");
    *W_out = 0.0;
    if (rounds_out) *rounds_out = 0;
    if (n == 1) return FAMST_OK;
    if (!tu || !tv || !tw) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    ST(check_points(ctx, X, n, d));
    ST(sync_status(ctx));
    const bool x3 = prec == FAMST_PREC_BF16X3;
    const bool tc = prec != FAMST_PREC_FP32 && knn_tc_supported(n, d, 1, x3);
    Arena ar;
    ST(ensure_ws(ctx, 1, emst_workspace(n, d, tc, x3, ctx->num_sms) + tree_weight_workspace(n), ar));
    Exec ex = exec_of(ctx);
    int64_t got = 0, unc = 0;
    int rounds = 0;
    ST(emst_exact(ex, ar, X, n, d, tc, x3, vec4_ok(X, d), MstOut{tu, tv, tw}, &got, &rounds, &unc,
                  ctx->pinned + PIN_KNN, ctx->pinned + PIN_MST));
    ST(sync_status(ctx));
    if (got != n - 1) return fail(ctx, FAMST_ERR_TIMEOUT, "Boruvka stopped before n - 1 edges");
    if (rounds_out) *rounds_out = rounds;
    ST(tree_weight(ex, ar, nullptr, 0, false, tu, tv, tw, n - 1, ctx->dW));
    double W[2];
    CK(cudaMemcpyAsync(W, ctx->dW, 16, cudaMemcpyDeviceToHost, ctx->stream));
    ST(sync_status(ctx));
    *W_out = W[0];
    return FAMST_OK;
}

famst_status famst_tree_weight(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                               const int32_t *tu, const int32_t *tv, const float *tw, int64_t m,
                               double *W, double *W64) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!W || !W64 || m < 0) return fail(ctx, FAMST_ERR_INVALID_ARG, "bad argument");
    if (m > 0 && (!tu || !tv || !tw || !X)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    Exec ex = exec_of(ctx);
    if (m > 0) {
        FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, m, 256), 256, 0, tu, m, n, 0, ctx->dstatus);
        FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, m, 256), 256, 0, tv, m, n, 0, ctx->dstatus);
    }
    ST(sync_status(ctx));
    Arena ar;
    ST(ensure_ws(ctx, 1, tree_weight_workspace(m), ar));
    ST(tree_weight(ex, ar, X, d, vec4_ok(X, d), tu, tv, tw, m, ctx->dW));
    double w[2];
    CK(cudaMemcpyAsync(w, ctx->dW, 16, cudaMemcpyDeviceToHost, ctx->stream));
    ST(sync_status(ctx));
    *W = w[0];
    *W64 = w[1];
    return FAMST_OK;
}

famst_status famst_build(famst_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t k,
                         int32_t lambda, uint64_t seed, int32_t prec, int32_t max_iters,
                         int32_t *tu, int32_t *tv, float *tw, double *W_out,
                         famst_build_info *info) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!W_out) return fail(ctx, FAMST_ERR_INVALID_ARG, "W_out NULL");
    if (n > 1 && (!tu || !tv || !tw)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL tree array");
    if (!X || n < 1 || d < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "bad X/n/d");
    CK(cudaSetDevice(ctx->device));
    return build_impl(ctx, X, n, d, k, lambda, seed, prec, max_iters, BuildOut{tu, tv, tw}, W_out,
                      info);
}

famst_status famst_build_host(famst_ctx *ctx, const float *X_host, int64_t n, int32_t d,
                              int32_t k, int32_t lambda, uint64_t seed, int32_t prec,
                              int32_t max_iters, int32_t *tu_host, int32_t *tv_host,
                              float *tw_host, double *W_out, famst_build_info *info) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!W_out || !X_host) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL argument");
    if (n > 1 && (!tu_host || !tv_host || !tw_host)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL tree array");
    if (n < 1 || d < 1 || n >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_INVALID_ARG, "bad n/d");
    CK(cudaSetDevice(ctx->device));
    size_t bx = align256(size_t(n) * d * 4), bt = align256(size_t(n) * 4);
    Arena ar;
    ST(ensure_ws(ctx, 2, bx + 3 * bt, ar));
    char *buf = ar.base;
    float *Xd = reinterpret_cast<float *>(buf);
    int32_t *tu = reinterpret_cast<int32_t *>(buf + bx);
    int32_t *tv = reinterpret_cast<int32_t *>(buf + bx + bt);
    float *tw = reinterpret_cast<float *>(buf + bx + 2 * bt);
    famst_status s = FAMST_OK;
    if (cudaMemcpyAsync(Xd, X_host, size_t(n) * d * 4, cudaMemcpyHostToDevice, ctx->stream) !=
        cudaSuccess)
        s = cuda_fail(ctx, cudaGetLastError(), "copy X");
    if (s == FAMST_OK)
        s = build_impl(ctx, Xd, n, d, k, lambda, seed, prec, max_iters, BuildOut{tu, tv, tw}, W_out,
                       info);
    if (s == FAMST_OK && n > 1) {
        size_t b = size_t(n - 1) * 4;
        if (cudaMemcpyAsync(tu_host, tu, b, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(tv_host, tv, b, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(tw_host, tw, b, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            s = cuda_fail(ctx, cudaGetLastError(), "copy tree");
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && s == FAMST_OK)
        s = cuda_fail(ctx, cudaGetLastError(), "synchronise");
    return s;
}

static famst_status batch_results(famst_ctx *ctx, const BatchCache &c, double *W, int64_t *t_out,
                                  famst_batch_info *info) {
    const int64_t *w = c.host.words;
    const int st = int(w[3]);
    if (st & batch_status_capacity()) return fail(ctx, FAMST_ERR_CAPACITY, "edge capacity");
    if (st & STATUS_NONFINITE) return fail(ctx, FAMST_ERR_NONFINITE, "X holds NaN or Inf");
    if (st & STATUS_LOOP_LIMIT) return fail(ctx, FAMST_ERR_TIMEOUT, "a bounded device loop reached its limit");
    if (st & STATUS_REFINE_CAP) return fail(ctx, FAMST_ERR_NO_CONVERGENCE, "refinement reached max_iters");
    if (st & (STATUS_DISCONNECTED | STATUS_BAD_ID)) return fail(ctx, FAMST_ERR_DISCONNECTED, "forest incomplete");
    for (int b = 0; b < c.B; ++b) {
        if (W) W[b] = c.host.W[b];
        if (t_out) t_out[b] = c.host.cbase[b + 1] - c.host.cbase[b];
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->m = w[0];
        int sweeps = 0;
        for (int q = 0; q <= c.max_iters; ++q)
            if (c.host.hist[q]) sweeps = q + 1;
        info->refine_sweeps = sweeps;
        info->boruvka_rounds = int32_t(w[2]);
        info->uncertified_rows = c.plan.any_tc ? w[4] : 0;
        info->tensor_clouds = 0;
        for (int b = 0; b < c.B; ++b) info->tensor_clouds += c.plan.cl[b].use_tc;
        info->graph_kernels = int64_t(c.graph_kernels);
        info->tile_epilogue_warps = c.plan.any_tc ? c.plan.tc_epi : 0;
        info->tile_stages = c.plan.any_tc ? c.plan.tc_stages : 0;
    }
    return FAMST_OK;
}

famst_status famst_build_batched(famst_ctx *ctx, const float *X, const int64_t *offsets,
                                 const int32_t *dims, int32_t B, int32_t k, int32_t lambda,
                                 uint64_t seed, int32_t prec, int32_t max_iters, int32_t *tu,
                                 int32_t *tv, float *tw, double *W, int64_t *t_out,
                                 famst_batch_info *info) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!X || !offsets || !dims || B < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "bad batch");
    if (lambda < 1 || lambda > 32) return fail(ctx, FAMST_ERR_INVALID_ARG, "need 1 <= lambda <= 32");
    if (max_iters < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "need max_iters >= 1");
    if (prec == FAMST_PREC_FP8) return fail(ctx, FAMST_ERR_UNSUPPORTED, "FP8 tiles: kNN graph and build only");
    if (prec < 0 || prec > 2) return fail(ctx, FAMST_ERR_INVALID_ARG, "unknown precision");
    if (k < 1 || k > 64) return fail(ctx, FAMST_ERR_UNSUPPORTED, "batched builds need 1 <= k <= 64");
    if (offsets[0] != 0) return fail(ctx, FAMST_ERR_INVALID_ARG, "offsets[0] must be 0");
    int dmax = 0;
    for (int b = 0; b < B; ++b) {
        const int64_t nb = offsets[b + 1] - offsets[b];
        if (nb < int64_t(k) + 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "every cloud needs n_b >= k + 1");
        if (dims[b] < 1) return fail(ctx, FAMST_ERR_INVALID_ARG, "dims must be >= 1");
        dmax = dims[b] > dmax ? dims[b] : dmax;
    }
    const int64_t N = offsets[B];
    if (N * int64_t(k) >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "sum(n)*k must be < 2^31");
    if (dmax > 512) return fail(ctx, FAMST_ERR_UNSUPPORTED, "batched builds need d <= 512");
    if (!tu || !tv || !tw) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL tree array");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));  // inputs are ordered before the private stream
    BatchCache &c = ctx->batch;
    const bool hit = c.valid && c.exec && c.B == B && c.k == k && c.lambda == lambda &&
                     c.prec == prec && c.max_iters == max_iters && c.seed == seed &&
                     int(c.offsets.size()) == B + 1 &&
                     std::equal(c.offsets.begin(), c.offsets.end(), offsets) &&
                     std::equal(c.dims.begin(), c.dims.end(), dims);
    // the captured sequence works on its own buffers: copy the clouds in
    // before it and the trees out after it
    auto copy_in = [&]() {
        return cudaMemcpyAsync(c.plan.dev.Xin, X, size_t(c.plan.xoff.back()) * 4,
                               cudaMemcpyDeviceToDevice, ctx->bstream);
    };
    auto copy_out = [&]() {
        const size_t m = size_t(N - B);
        cudaError_t e = cudaSuccess;
        if (m > 0) {
            e = cudaMemcpyAsync(tu, c.plan.dev.out_u, m * 4, cudaMemcpyDeviceToDevice, ctx->bstream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(tv, c.plan.dev.out_v, m * 4, cudaMemcpyDeviceToDevice, ctx->bstream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(tw, c.plan.dev.out_w, m * 4, cudaMemcpyDeviceToDevice, ctx->bstream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->bstream);
        return e;
    };
    if (hit) {
        CK(copy_in());
        CK(cudaGraphLaunch(c.exec, ctx->bstream));
        CK(copy_out());
        ctx->launches += c.graph_kernels;
        famst_status s = batch_results(ctx, c, W, t_out, info);
        if (info) info->graph_replayed = 1;
        return s;
    }
    c.release();
    c.offsets.assign(offsets, offsets + B + 1);
    c.dims.assign(dims, dims + B);
    c.B = B; c.k = k; c.lambda = lambda; c.prec = prec; c.max_iters = max_iters; c.seed = seed;
    c.X = X; c.tu = tu; c.tv = tv; c.tw = tw;
    Exec ex{ctx->bstream, &ctx->launches, ctx->num_sms, ctx->dstatus};
    // first guess for the edge capacity: up to 48 components per cloud
    int64_t m_cap = 0;
    for (int b = 0; b < B; ++b) {
        int64_t tb = (offsets[b + 1] - offsets[b]) / (k + 1);
        tb = tb < 48 ? tb : 48;
        m_cap += int64_t(lambda) * tb * (tb - 1) / 2;
    }
    famst_status s = FAMST_OK;
    for (int attempt = 0; attempt < 2; ++attempt) {
        s = batch_plan(ex, offsets, dims, B, k, lambda, prec, max_iters, m_cap, &c.plan);
        if (s != FAMST_OK) return fail(ctx, s, "batch plan");
        Arena ar;
        ST(ensure_ws(ctx, 3, batch_workspace(c.plan), ar));
        ST(batch_bind(c.plan, ar.base, ar.cap, ctx->bstream));
        if (!c.host.W) {
            CK(cudaMallocHost(&c.host.W, size_t(B) * 8));
            CK(cudaMallocHost(&c.host.cbase, size_t(B + 1) * 4));
            CK(cudaMallocHost(&c.host.hist, size_t(max_iters + 1) * 4));
            CK(cudaMallocHost(&c.host.words, 8 * 8));
        }
        memset(c.host.words, 0, 64);
        CK(copy_in());
        s = batch_enqueue(ex, c.plan, ar.base, ar.cap, seed, &c.host);
        if (s != FAMST_OK) return fail(ctx, s, "batch enqueue");
        CK(copy_out());
        if ((int(c.host.words[3]) & batch_status_capacity()) && attempt == 0) {
            m_cap = c.host.words[0] + c.host.words[0] / 4 + 1;  // the device reported what it needs
            continue;
        }
        break;
    }
    s = batch_results(ctx, c, W, t_out, info);
    if (s != FAMST_OK) return s;
    // tile shape of the tensor pass, timed on this batch's prepared operands
    s = batch_tune_tiles(ex, c.plan);
    if (s != FAMST_OK) return fail(ctx, s, "batch tile tuning");
    // capture the same sequence once; later calls with this key replay it
    unsigned long long counted = 0;
    Exec cap_ex{ctx->bstream, &counted, ctx->num_sms, ctx->dstatus};
    CK(cudaStreamBeginCapture(ctx->bstream, cudaStreamCaptureModeRelaxed));
    famst_status se = batch_enqueue(cap_ex, c.plan, ctx->ws[3], ctx->ws_cap[3], seed, &c.host);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(ctx->bstream, &g);
    if (se != FAMST_OK || ee != cudaSuccess || !g) {
        // the eager run's results stand; no graph is cached (reason kept)
        snprintf(ctx->err, sizeof(ctx->err), "graph capture failed: %s / %s",
                 famst_error_string(se), cudaGetErrorString(ee));
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (info) info->graph_kernels = -1;
        return FAMST_OK;
    }
    cudaError_t ei = cudaGraphInstantiate(&c.exec, g, 0);
    if (ei != cudaSuccess) {
        snprintf(ctx->err, sizeof(ctx->err), "graph instantiation failed: %s", cudaGetErrorString(ei));
        cudaGraphDestroy(g);
        cudaGetLastError();
        c.exec = nullptr;
        if (info) info->graph_kernels = -1;
        return FAMST_OK;
    }
    c.graph = g;
    c.graph_kernels = counted;
    c.valid = true;
    if (info) {
        info->graph_kernels = int64_t(counted);
        info->tile_epilogue_warps = c.plan.any_tc ? c.plan.tc_epi : 0;
        info->tile_stages = c.plan.any_tc ? c.plan.tc_stages : 0;
    }
    return FAMST_OK;
}

famst_status famst_mst_backward(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                                const int32_t *tu, const int32_t *tv, int64_t m, float gW,
                                float *gX) {
    if (!ctx) return FAMST_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (!gX || m < 0) return fail(ctx, FAMST_ERR_INVALID_ARG, "bad argument");
    if (m > 0 && (!tu || !tv)) return fail(ctx, FAMST_ERR_INVALID_ARG, "NULL tree array");
    if (2 * m >= (int64_t(1) << 31)) return fail(ctx, FAMST_ERR_UNSUPPORTED, "too many edges");
    CK(cudaSetDevice(ctx->device));
    ST(reset_status(ctx));
    if (n < 1 || (n * int64_t(d)) >= (int64_t(1) << 40)) return fail(ctx, FAMST_ERR_INVALID_ARG, "bad n/d");
    ST(check_points(ctx, X, n, d));
    Exec ex = exec_of(ctx);
    if (m > 0) {
        FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, m, 256), 256, 0, tu, m, n, 0, ctx->dstatus);
        FAMST_LAUNCH(ex, check_ids_kernel, grid_cap(ctx, m, 256), 256, 0, tv, m, n, 0, ctx->dstatus);
    }
    ST(sync_status(ctx));
    Arena ar;
    ST(ensure_ws(ctx, 1, mst_backward_workspace(n, m), ar));
    ST(mst_backward(ex, ar, X, n, d, vec4_ok(X, d), tu, tv, m, gW, gX));
    return sync_status(ctx);
}

}  // extern "C"
