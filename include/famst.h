/*
 * famst.h -- C ABI of the GB300 (sm_103a) FAMST library.
 *
 * FAMST (Almansoori & Telek) builds an approximate Euclidean minimum
 * spanning tree of n points in d dimensions in three phases (Algorithm 1):
 *   Phase 1  kNN graph of the points                       famst_knn_graph
 *   Phase 2  connected components of the undirected graph  famst_components
 *            (Algorithm 2) and lambda inter-component edges
 *            per component pair (Algorithm 3)              famst_connect
 *   Phase 3  neighbourhood refinement of those edges,
 *            repeated until no edge changes (Algorithm 4)  famst_refine
 *   then     Kruskal-equivalent MST of kNN edges + E       famst_mst
 * famst_build runs all of it. famst_mst_backward differentiates the tree
 * weight with respect to the points; famst_build_batched runs many clouds.
 * famst_components_noalloc labels components without any allocation;
 * famst_emst_exact computes the exact EMST T* that Eq. 1 compares with.
 *
 * Conventions for every call:
 *  - Pointers are DEVICE pointers owned by the caller unless the argument
 *    is documented as HOST. Nothing is freed or retained by the library.
 *  - X is row-major float32, n rows of d contiguous floats (stride d).
 *  - Vertex ids are int32 (n < 2^31); n*k must be < 2^31.
 *  - Work is enqueued on the context's stream (famst_set_stream; default
 *    is the legacy default stream). Calls that return a value through a
 *    HOST pointer synchronise that stream before returning; the others
 *    return once the work is enqueued.
 *  - The library owns one device workspace per context; it grows on demand
 *    (cudaMalloc) and is freed by famst_destroy. A context must not be used
 *    from two host threads at once.
 *  - Errors: every call returns a famst_status. On error the outputs are
 *    undefined but the context stays usable. Nothing aborts.
 *
 * Distances. Every distance the library computes, stores or compares is the
 * canonical FP32 Euclidean distance: 32 partial sums
 *     p_l = 0; for t = l, l+32, l+64, ... < d: delta = x[t] - y[t];
 *                                              p_l = fmaf(delta, delta, p_l)
 * combined by the butterfly o = 16, 8, 4, 2, 1: p_l = p_l + p_(l xor o)
 * (all l at once), then w = sqrtf(p_0); every operation IEEE
 * round-to-nearest. It is the order a 32-lane warp evaluates naturally, and
 * it is symmetric bit for bit. Orders: neighbours of a row by (w, id);
 * edges by (w, min id, max id). Weights of trees are summed in FP64.
 */
#ifndef FAMST_H
#define FAMST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t famst_status;

#define FAMST_OK                  0
#define FAMST_ERR_INVALID_ARG    -1  /* null pointer, bad size, k or lambda out of range */
#define FAMST_ERR_CAPACITY       -2  /* output buffer too small; the required size is returned */
#define FAMST_ERR_NO_CONVERGENCE -3  /* refinement still changing after max_iters sweeps */
#define FAMST_ERR_TIMEOUT        -4  /* a bounded device loop gave up */
#define FAMST_ERR_CUDA           -5  /* a CUDA runtime call failed */
#define FAMST_ERR_OOM            -6  /* workspace allocation failed */
#define FAMST_ERR_UNSUPPORTED    -7  /* size or mode this build does not handle */
#define FAMST_ERR_NONFINITE      -8  /* X holds a NaN or an infinity */
#define FAMST_ERR_DISCONNECTED   -9  /* famst_mst: the candidate graph is not connected */

/* Distance-tile precision for Phase 1 (famst_knn_graph, famst_build).
 * Every precision returns the exact kNN under the canonical distance:
 * the tiles only choose candidates, which are re-ranked on canonical
 * distances; a row whose candidate set cannot be certified from the tile's
 * error bound is recomputed by the FP32 tiles, and a row those cannot
 * certify either (ties at the k-th distance) by an exact warp-per-row brute
 * force on canonical distances. */
#define FAMST_PREC_FP32   0  /* SIMT FP32 tiles (k + 8 candidates by a fast FP32 sum) */
#define FAMST_PREC_BF16   1  /* tcgen05 BF16 tiles (x.y on tensor cores), FP32 re-rank */
#define FAMST_PREC_BF16X3 2  /* tcgen05 BF16 hi/lo split, 3 products, FP32 re-rank */
/* tcgen05 E4M3 tiles (kind::f8f6f4), each centred row scaled by a power of
 * two to the E4M3 range, FP32 re-rank. famst_knn_graph and famst_build
 * only (famst_emst_exact and famst_build_batched return UNSUPPORTED); no
 * tile pruning. Its error bound is ~2^-4 relative, so on clouds whose k-th
 * and (k+8)-th neighbour distances are closer than that most rows fall back
 * to the FP32 tiles: the result stays exact, the time does not. */
#define FAMST_PREC_FP8    3

typedef struct famst_ctx famst_ctx;

/* Per-build statistics, filled by famst_build* when the HOST pointer is
 * not NULL. Times are CUDA-event milliseconds per stage on the context
 * stream. */
typedef struct famst_build_info {
    int64_t t;                /* components of the kNN graph (Alg. 2) */
    int64_t m;                /* inter-component edges, lambda*t*(t-1)/2 (Alg. 3) */
    int32_t refine_sweeps;    /* sweeps of Alg. 4 until |Delta| = 0, the last included */
    int32_t boruvka_rounds;
    int64_t first_delta;      /* |Delta| of the first sweep */
    int64_t uncertified_rows; /* reduced-precision rows recomputed in FP32 */
    double  W;                /* sum of the FP32 tree weights, in FP64 */
    double  W64;              /* tree weight with every edge recomputed in FP64 */
    double  ms_knn, ms_components, ms_connect, ms_refine, ms_mst, ms_total;
    double  knn_tile_fraction; /* (query, key) tile pairs Phase 1 computed / all pairs */
    int64_t refine_distance_evals; /* candidate distances Algorithm 4 evaluated */
    int64_t refine_canonical_evals; /* of which the canonical distance decided */
    int32_t refine_filter;    /* candidate filter of Algorithm 4's kernel: -1 no refinement
                                 (t = 1), 0 none (canonical distance per candidate),
                                 1 FP32 grouped sums, 2 BF16 dot products on the tensor
                                 cores (mma.sync); survivors of a filter are decided on
                                 canonical distances, so the result is the same */
    int32_t knn_iters;        /* NN-Descent iterations of Phase 1 (0: exact tiles) */
    /* CUDA-event milliseconds of single kernels (0 when the kernel did not
     * run): the tcgen05 distance tiles of Phase 1's main pass, the
     * canonical re-rank with its certificate, Algorithm 3's kernel and
     * Algorithm 4's kernel */
    double  ms_knn_tiles, ms_rerank, ms_connect_kernel, ms_refine_kernel;
    /* rows Algorithm 4's kernels read (filter 2 only, 0 otherwise): candidate
     * BF16 rows staged in shared memory, and rows of fixed points (one per
     * scan); each canonical evaluation reads two FP32 rows */
    int64_t refine_rows_staged, refine_fixed_rows;
} famst_build_info;

/* ------------------------------------------------------------ context */

/* Create a context on CUDA device `device`. *out receives it. */
famst_status famst_create(famst_ctx **out, int device);
/* Free the context and its workspace. NULL is accepted. */
famst_status famst_destroy(famst_ctx *ctx);
/* Enqueue all later work on `stream` (a cudaStream_t; NULL = legacy default). */
famst_status famst_set_stream(famst_ctx *ctx, void *stream);
/* Phase 1 tile pruning (exact either way): 1 = on where the shape allows it
 * (the default), 0 = every (query, key) tile pair is computed. With pruning
 * the points are partitioned into cells around evenly spaced pivots and a
 * query tile skips the key tiles that a triangle-inequality bound places
 * beyond an upper bound on its rows' k-th neighbour distance; the
 * certificate covers the skipped keys, so the kNN graph is unchanged. */
famst_status famst_set_knn_pruning(famst_ctx *ctx, int32_t enable);
/* *bytes (HOST) = device workspace a famst_build (or famst_build_host,
 * whose device copies of X and the tree come on top) of this shape needs
 * when its kNN graph has at most t_max components (Algorithm 2's t; the
 * connect and refine workspace grows with lambda t (t - 1) / 2). The
 * context grows its workspace to that size on first use (cudaMalloc) and
 * keeps it; a caller that wants to allocate up front runs one build of the
 * largest shape first. Depends on the context's pruning setting. Errors:
 * INVALID_ARG (bad shape, 1 <= t_max <= n), UNSUPPORTED (as famst_build). */
famst_status famst_workspace_query(famst_ctx *ctx, int64_t n, int32_t d, int32_t k,
                                   int32_t lambda, int64_t t_max, int32_t prec,
                                   int32_t max_iters, size_t *bytes);
/* Connect step of famst_build / famst_build_host: FAMST_CONNECT_RANDOM
 * (Algorithm 3, the default) or FAMST_CONNECT_NEAREST (famst_connect_nearest;
 * the rest of Algorithm 1 is unchanged). */
#define FAMST_CONNECT_RANDOM  0
#define FAMST_CONNECT_NEAREST 1
famst_status famst_set_connect_mode(famst_ctx *ctx, int32_t mode);
/* Iteration limit of the library's bounded loops: each find and hook loop
 * of the union-find (Algorithm 2), the pointer jumping of every Boruvka
 * round, and the number of Boruvka rounds (at most 64). A loop that reaches
 * the limit makes the call return FAMST_ERR_TIMEOUT instead of a result; the
 * context stays usable. 0 (the default) restores the built-in limits
 * (2^22 steps, 64 rounds), which no valid input reaches. */
famst_status famst_set_loop_limit(famst_ctx *ctx, int32_t limit);
/* Static string naming a status code. */
const char *famst_error_string(famst_status status);
/* Detail of the last error on this context (static storage in ctx). */
const char *famst_last_error(const famst_ctx *ctx);
/* Number of kernels this context has launched so far. */
uint64_t famst_launch_count(const famst_ctx *ctx);
/* Workspace bytes currently held by the context. */
size_t famst_workspace_bytes(const famst_ctx *ctx);

/* ------------------------------------------------------- Phase 1: kNN
 * GetANNs of Algorithm 1, realised as the exact kNN by brute force over
 * distance tiles: for each row i, the k smallest (w(i,j), j) with j != i,
 * ascending. nbr[i*k + r] and dist[i*k + r] (n x k each, device).
 * Requires 1 <= k <= n-1 and k <= 128. prec: FAMST_PREC_*. Errors:
 * INVALID_ARG, NONFINITE, UNSUPPORTED (tensor precisions need d <= 512). */
famst_status famst_knn_graph(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                             int32_t k, int32_t prec, int32_t *nbr, float *dist);

/* --------------------------------------- Phase 1 alternative: NN-Descent
 * GetANNs of Algorithm 1 as the paper runs it: an approximate kNN graph by
 * NN-Descent (Dong, Charikar and Li, WWW 2011; the paper's Phase 1 library
 * implements it, Sec. 2 and 3). Each step is a set operation, so the
 * result is deterministic for a seed:
 *   start  B[v] = the first k distinct ids among the draws
 *          u = (r0 (n-1)) >> 32 (u += 1 if u >= v), r0 the first word of
 *          Philox4x32-10(counter (v, r, 0, 1), key (seed_lo, seed_hi)),
 *          r = 0 .. 8k-1, then the smallest unused ids; or init_nbr's row
 *          (device, n x k distinct ids != v; NULL = draw); all entries new;
 *   each iteration it = 0, 1, ...:
 *     new[v] / old[v] = the S candidates smallest in (pr, u), pr = r0 of
 *          Philox(counter (v, u, it, 2)), among the ids of B[v] flagged
 *          new / old and the ids u whose B[u] holds v flagged new / old;
 *          the new entries of B[v] that made new[v] become old;
 *     every pair {a, b} of new[v] x new[v] and new[v] x old[v] (a != b)
 *          proposes b to B[a] and a to B[b] with the canonical w(a, b);
 *     B[a] = the k smallest distinct (w, id) of B[a] and its proposals,
 *          added entries new; c = the number of entries added;
 *   stop after an iteration with c = 0 or c < delta n k, or max_iters.
 * nbr / dist (device, n x k) receive the lists, (w, id) ascending;
 * *iters_out (HOST, may be NULL) = iterations run; updates and pairs (HOST
 * arrays of max_iters, may be NULL) = c and the pairs the joins evaluated
 * (C(|new[v]|, 2) + |new[v] x old[v]| over v, less pairs a = b) per
 * iteration. Requires 1 <= k <= 32,
 * k <= n-1, 1 <= S <= 32, max_iters >= 0, delta >= 0. Errors: INVALID_ARG
 * (also a bad init_nbr row), NONFINITE, UNSUPPORTED (2 S rows of d floats
 * beyond 200 KB of shared memory). Synchronises once per iteration. */
famst_status famst_knn_nndescent(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                                 int32_t k, int32_t S, int32_t max_iters, double delta,
                                 uint64_t seed, const int32_t *init_nbr, int32_t *nbr,
                                 float *dist, int32_t *iters_out, int64_t *updates,
                                 int64_t *pairs);

/* Phase 1 of famst_build / famst_build_host: FAMST_KNN_EXACT (the exact
 * tiles at the build's precision, the default) or FAMST_KNN_NNDESCENT
 * (famst_knn_nndescent with the build's seed and these S (0: min(k, 32)),
 * max_iters and delta; the build's prec is then unused). */
#define FAMST_KNN_EXACT      0
#define FAMST_KNN_NNDESCENT  1
famst_status famst_set_knn_method(famst_ctx *ctx, int32_t method, int32_t S, int32_t max_iters,
                                  double delta);

/* ------------------------------------------------ Phase 2a: Algorithm 2
 * Connected components of the undirected graph G built from nbr (n x k):
 * comp[v] (device, n) = index of v's component, components numbered in
 * ascending order of their smallest vertex id -- the order in which the
 * depth-first search of Algorithm 2 discovers them. *t_out (HOST) = t.
 * Synchronises. */
famst_status famst_components(famst_ctx *ctx, const int32_t *nbr, int64_t n, int32_t k,
                              int32_t *comp, int64_t *t_out);

/* ------------------------------------------------ Phase 2b: Algorithm 3
 * For every component pair i < j (i outer, j inner) draw lambda^2 samples
 * s = 0..lambda^2-1 with Philox4x32-10 (counter (s, p_lo, p_hi, 0),
 * key (seed_lo, seed_hi), p = i*t + j):
 *     u = C_i[(r0 * |C_i|) >> 32],  v = C_j[(r1 * |C_j|) >> 32]
 * where C_c lists component c's vertices by ascending id, and keep the
 * lambda samples with the smallest (w(u,v), s), ascending. Edge
 * e = (pair rank)*lambda + r is (eu, ev, ew) with eu in C_i, ev in C_j and
 * (eci, ecj) = (i, j). comp/t as returned by famst_components.
 * capacity = length of the five edge arrays (device); *m_out (HOST)
 * receives lambda*t*(t-1)/2, also when it exceeds capacity (CAPACITY).
 * 1 <= lambda <= 32. Synchronises. */
famst_status famst_connect(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                           const int32_t *comp, int64_t t, int32_t lambda, uint64_t seed,
                           int32_t *eu, int32_t *ev, float *ew, int32_t *eci, int32_t *ecj,
                           int64_t capacity, int64_t *m_out);

/* ------------------------------- Phase 2b variant: the nearest pairs
 * The variant of Algorithm 3 that joins components by their nearest pairs
 * ("the lambda nearest cross-component edges", Sec. 3 on joining the
 * components): for every component pair i < j (i outer, j inner), the
 * lambda pairs (u in C_i, v in C_j) with the smallest canonical distance
 * under the order (w, min id, max id), ascending, over all |C_i| |C_j|
 * pairs. A pair with fewer than lambda cross pairs repeats its farthest
 * pair. Same arguments, layout and errors as famst_connect (no seed);
 * 1 <= d <= 256 (UNSUPPORTED beyond). The work is all cross pairs (about
 * n^2 / 2 distance evaluations on the tensor cores, filtered by rigorous
 * bounds and decided on canonical distances). Synchronises. */
famst_status famst_connect_nearest(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                                   const int32_t *comp, int64_t t, int32_t lambda,
                                   int32_t *eu, int32_t *ev, float *ew, int32_t *eci,
                                   int32_t *ecj, int64_t capacity, int64_t *m_out);

/* ------------------------------------------------- Phase 3: Algorithm 4
 * Repeat the refinement sweep of Algorithm 4 over the m edges in place
 * until no edge changes, at most max_iters sweeps. One sweep moves u to
 * the neighbour u' in G[u] (same component) minimising w(u', v) when that
 * is strictly smaller, then v likewise against the new u. Edges are
 * independent, so each is iterated to its own fixed point; the result
 * equals that of global sweeps. *sweeps_out (HOST) = number of sweeps
 * including the final one without change; delta_hist (HOST, may be NULL,
 * max_iters entries) receives |Delta| of each sweep. Errors:
 * NO_CONVERGENCE when an edge still changed in sweep max_iters.
 * Synchronises. */
famst_status famst_refine(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                          const int32_t *nbr, int32_t k, const int32_t *comp,
                          int32_t *eu, int32_t *ev, float *ew,
                          const int32_t *eci, const int32_t *ecj, int64_t m,
                          int32_t max_iters, int32_t *sweeps_out, int64_t *delta_hist);

/* ------------------------------------------------------------- MST
 * Minimum spanning tree of the graph made of the kNN edges {i, nbr[i*k+r]}
 * weighted dist[i*k+r] and the m edges (eu, ev, ew), under the total
 * order (w, min id, max id) -- the tree Kruskal's algorithm returns --
 * computed by Boruvka rounds. tu/tv/tw (device, n-1 each) receive the
 * edges as (min id, max id, w) in the order (round, component) in which
 * they were found. *W_out (HOST) = sum of tw in FP64. Errors:
 * DISCONNECTED. Synchronises. */
famst_status famst_mst(famst_ctx *ctx, int64_t n, const int32_t *nbr, const float *dist,
                       int32_t k, const int32_t *eu, const int32_t *ev, const float *ew,
                       int64_t m, int32_t *tu, int32_t *tv, float *tw, double *W_out);

/* FP64 weights of a tree: *W (HOST) = sum of tw in FP64 (fixed-order
 * reduction); *W64 (HOST) = sum over edges of the distance recomputed in
 * FP64 from X. Synchronises. */
famst_status famst_tree_weight(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                               const int32_t *tu, const int32_t *tv, const float *tw,
                               int64_t m, double *W, double *W64);

/* ----------------------------------------------------- whole build
 * Algorithm 1 end to end on device data: kNN (prec), components,
 * connect (lambda, seed), refine (max_iters), MST. tu/tv/tw: n-1 each
 * (device). *W_out and *info (HOST; info may be NULL). Synchronises. */
famst_status famst_build(famst_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t k,
                         int32_t lambda, uint64_t seed, int32_t prec, int32_t max_iters,
                         int32_t *tu, int32_t *tv, float *tw, double *W_out,
                         famst_build_info *info);

/* famst_build with X, tu, tv, tw all in HOST memory: copies X in and the
 * tree out on the context stream (pinned memory makes the copies fast). */
famst_status famst_build_host(famst_ctx *ctx, const float *X_host, int64_t n, int32_t d,
                              int32_t k, int32_t lambda, uint64_t seed, int32_t prec,
                              int32_t max_iters, int32_t *tu_host, int32_t *tv_host,
                              float *tw_host, double *W_out, famst_build_info *info);

/* ----------------------------------------------------- many clouds
 * Builds of B independent clouds in one call. X (device) holds the clouds
 * back to back: cloud b is n_b = offsets[b+1] - offsets[b] rows of dims[b]
 * floats (offsets: HOST, B+1 entries, offsets[0] = 0; dims: HOST, B).
 * Cloud b's result is bit-identical to famst_build of that cloud alone with
 * seed + b. Every phase runs once over the whole batch (a fixed sequence of
 * launches whose data-dependent counts stay on the device); the first call
 * for a given shape, parameters and pointers runs it and captures it in a
 * CUDA graph, later identical calls replay the graph. Phase 1 uses the
 * tensor tiles or the FP32 tiles per cloud, as an autotuner measured
 * faster on this device for that cloud's (d, n) class (cached per process;
 * appended to the file named by FAMST_AUTOTUNE_CACHE when set).
 * tu/tv/tw (device, offsets[B] - B entries): cloud b's n_b - 1 tree edges at
 * [offsets[b] - b, offsets[b+1] - b - 1), as cloud-local ids in
 * (round, component) order. W (HOST, B): FP64 tree weight per cloud; t_out
 * (HOST, B, may be NULL): components of each cloud's kNN graph.
 * Requires n_b >= k + 1, 1 <= k <= 64, dims <= 512. Synchronises. */
typedef struct famst_batch_info {
    int64_t m;                /* inter-component edges of all clouds */
    int32_t refine_sweeps;    /* largest sweep count of any cloud */
    int32_t boruvka_rounds;
    int64_t uncertified_rows; /* tensor-tile rows recomputed in FP32 */
    int32_t tensor_clouds;    /* clouds whose Phase 1 ran on the tensor tiles */
    int32_t graph_replayed;   /* 1 if this call replayed a captured graph */
    int64_t graph_kernels;    /* kernels in the captured sequence */
    int32_t tile_epilogue_warps;  /* tile shape the autotuner chose for the tensor pass */
    int32_t tile_stages;          /* (0 when no cloud used the tensor tiles) */
} famst_batch_info;

famst_status famst_build_batched(famst_ctx *ctx, const float *X, const int64_t *offsets,
                                 const int32_t *dims, int32_t B, int32_t k, int32_t lambda,
                                 uint64_t seed, int32_t prec, int32_t max_iters, int32_t *tu,
                                 int32_t *tv, float *tw, double *W, int64_t *t_out,
                                 famst_batch_info *info);

/* -------------------------------------------------------- backward
 * Gradient of W = sum over tree edges of ||x_u - x_v|| with the tree held
 * fixed: gX[i] = gW * sum over edges e at i of (x_i - x_other)/w_e, where
 * w_e is the canonical distance; an edge with w_e = 0 contributes 0. Each
 * vertex sums its edges in ascending edge index, so the result is
 * deterministic. gX: n x d (device), overwritten. */
famst_status famst_mst_backward(famst_ctx *ctx, const float *X, int64_t n, int32_t d,
                                const int32_t *tu, const int32_t *tv, int64_t m,
                                float gW, float *gX);

/* ------------------------------------------------------ exact EMST
 * The exact Euclidean MST T* of the complete graph on the n points: the
 * reference tree of the relative error (W - W*) / W* of Eq. 1, computed on
 * the GPU so it is available at sizes where an O(n^2) CPU Prim is not.
 * Boruvka on the complete graph: each round finds every point's nearest
 * neighbour outside its current component with an exact masked 1-NN pass
 * (the Phase 1 distance tiles, precision `prec`, with the same FP32
 * re-rank and certificate), then hooks every component by its minimum
 * outgoing edge under (w, min id, max id). The tree is the unique MST
 * under that order, identical to Prim's or Kruskal's on the complete graph
 * with canonical FP32 weights.
 * X (device, n x d). tu/tv/tw (device, n - 1): tree edges in (round,
 * component) order, tu < tv. *W_out (HOST): FP64 sum of tw; *rounds_out
 * (HOST, may be NULL): Boruvka rounds. Requires n >= 1 (n = 1: empty
 * tree), 1 <= d. Cost: one all-pairs distance pass per round, at most
 * ceil(log2 n) rounds. Synchronises. */
famst_status famst_emst_exact(famst_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t prec,
                              int32_t *tu, int32_t *tv, float *tw, double *W_out,
                              int32_t *rounds_out);

/* ----------------------------------------- allocation-free components
 * The paper has no counterpart to this call: it is an interface variant of
 * famst_components for callers that cannot allocate device memory -- for
 * example a host application that reserves all GPU memory for its own
 * pool allocator at start-up, or a latency-critical loop that cannot
 * tolerate the device-wide synchronisation cudaMalloc and cudaFree imply.
 * It needs no famst_ctx and never calls cudaMalloc, cudaFree or any
 * allocating library routine.
 *
 * Same result as famst_components: comp[v] (device, n) = component index
 * in ascending order of the components' smallest ids; *t_dev (DEVICE
 * int32) = t, or -1 when nbr holds an id outside [0, n) or a self-loop.
 * Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default) on
 * the calling thread's current device; the call returns without
 * synchronising.
 *
 * Scratch: one static device array of about 8.4 MB (2 * FAMST_NOALLOC_MAX_N
 * int32 plus small tables), present on every GPU that loads this library
 * until the process exits. n > FAMST_NOALLOC_MAX_N returns
 * FAMST_ERR_UNSUPPORTED; 1 <= k <= n-1 and n*k < 2^31 are required.
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, which allocates nothing; nothing is cached, so
 * calls stay valid after cudaDeviceReset). The first call in a context may
 * load the module, so make it before any stream capture. Every call on a
 * device shares the array and leaves its contents
 * behind (each call initialises what it reads); calls whose work overlaps
 * on the GPU race on it, so serialise them (one stream, or events). */
#define FAMST_NOALLOC_MAX_N (1 << 20)
famst_status famst_components_noalloc(const int32_t *nbr, int64_t n, int32_t k,
                                      int32_t *comp, int32_t *t_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FAMST_H */
