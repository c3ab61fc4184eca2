// MST extraction (the Kruskal step at the end of Algorithm 1), the FP64
// tree weight, and the gradient of the tree weight.
//
// Kruskal's algorithm on a graph whose edges are totally ordered returns
// the unique MST under that order; Boruvka's algorithm returns the same
// tree (cut property). The device runs edge-centric Boruvka rounds under
// the order (w, min id, max id):
//   1. every edge joining two components offers (w, min id) to both
//      components with a 64-bit atomicMin, then, among the edges that
//      matched the winner, the max id with a second atomicMin: together
//      the lexicographic minimum of the 96-bit key, found without sorting;
//   2. each component hooks to the component across its minimum edge;
//      two components that chose the same edge form the only possible
//      cycle and the smaller id stays root; the others record their edge;
//   3. pointer jumping makes every component point to its new root and the
//      vertices are relabelled.
// The edge set is the kNN graph (edge i -> nbr[i*k + r], weight
// dist[i*k + r]; both directions of a mutual pair are the same edge) plus
// the m inter-component edges. Tree edges are written in the order
// (round, component id), which is deterministic.
#include <cuda_runtime.h>

#include "famst_internal.cuh"

namespace famst {
namespace {

constexpr int JUMP_LIMIT = 1 << 22;

struct EdgeSrc {
    const int32_t *nbr;
    const float *dist;
    int k;
    int64_t nk;
    const int32_t *eu, *ev;
    const float *ew;
    int64_t m;
    const int64_t *m_dev;   // optional device-side count of E edges (<= m)
    __device__ __forceinline__ int64_t total() const {
        return nk + (m_dev ? (*m_dev < m ? *m_dev : m) : m);
    }
    __device__ __forceinline__ void get(int64_t e, int &a, int &b, float &w) const {
        if (e < nk) {
            a = int(e / k);
            b = nbr[e];
            w = dist[e];
        } else {
            int64_t q = e - nk;
            a = eu[q];
            b = ev[q];
            w = ew[q];
        }
    }
};

__global__ void bv_init_kernel(int32_t *comp, int64_t n) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = int32_t(v);
}

// Lanes of a warp whose edges end in the same component first take the
// minimum of their keys (match + two 32-bit reductions: the weight bits,
// then the smaller id among the lanes holding the minimum weight), and one
// lane per component issues the atomic: in the late rounds, where few
// components remain, millions of edges would otherwise hit the same few
// addresses. The result is the same minimum.
__device__ __forceinline__ void warp_min_to(unsigned long long *__restrict__ best, int c,
                                            unsigned long long key, int lane) {
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const unsigned hi = unsigned(key >> 32), lo = unsigned(key);
    const unsigned mhi = __reduce_min_sync(peers, hi);
    const unsigned mlo = __reduce_min_sync(peers, hi == mhi ? lo : 0xffffffffu);
    if (c >= 0 && lane == __ffs(peers) - 1)
        atomicMin(best + c, (uint64_t(mhi) << 32) | mlo);
}

__global__ void bv_min1_kernel(EdgeSrc es, const int32_t *__restrict__ comp,
                               unsigned long long *__restrict__ best1, const int *__restrict__ done,
                               int32_t *__restrict__ ou = nullptr, int32_t *__restrict__ ov = nullptr,
                               float *__restrict__ ow = nullptr,
                               unsigned long long *__restrict__ ocount = nullptr) {
    if (done && *done) return;
    const int64_t total = es.total();
    const int lane = threadIdx.x & 31;
    // whole warps step together (the warp-wide reductions need every lane)
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e0 = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); e0 < total;
         e0 += stride) {
        const int64_t e = e0 + lane;
        int a = 0, b = 0, ca = -1, cb = -1;
        float w = 0.0f;
        if (e < total) {
            es.get(e, a, b, w);
            ca = comp[a];
            cb = comp[b];
        }
        const bool inter = e < total && ca != cb;
        const unsigned long long key1 =
            (uint64_t(__float_as_uint(w)) << 32) | uint32_t(a < b ? a : b);
        warp_min_to(best1, inter ? ca : -1, key1, lane);
        warp_min_to(best1, inter ? cb : -1, key1, lane);
        if (ocount) {   // append the edges between components, one atomic per warp
            const unsigned bal = __ballot_sync(0xffffffffu, inter);
            if (bal) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(ocount, (unsigned long long)__popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (inter) {
                    const unsigned long long idx = base + __popc(bal & ((1u << lane) - 1u));
                    ou[idx] = a;
                    ov[idx] = b;
                    ow[idx] = w;
                }
            }
        }
    }
}

__global__ void bv_min2_kernel(EdgeSrc es, const int32_t *__restrict__ comp,
                               const unsigned long long *__restrict__ best1,
                               unsigned int *__restrict__ best2, const int *__restrict__ done) {
    if (done && *done) return;
    int64_t total = es.total();
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        int a, b;
        float w;
        es.get(e, a, b, w);
        int ca = comp[a], cb = comp[b];
        if (ca == cb) continue;
        unsigned long long key1 = (uint64_t(__float_as_uint(w)) << 32) | uint32_t(a < b ? a : b);
        unsigned int mx = unsigned(a < b ? b : a);
        if (best1[ca] == key1) atomicMin(best2 + ca, mx);
        if (best1[cb] == key1) atomicMin(best2 + cb, mx);
    }
}

// First round (every vertex its own component): a vertex's minimum incident
// edge under (w, min, max) is its first kNN entry -- the list is the exact
// top-k by (w, id), so no edge at v, kNN or inter-component, is lighter, and
// at equal w the smallest id comes first. No edge scan is needed.
__global__ void bv_first_kernel(const int32_t *__restrict__ nbr, const float *__restrict__ dist,
                                int k, int64_t n, unsigned long long *__restrict__ best1,
                                unsigned int *__restrict__ best2) {
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int j = nbr[v * k];
    if (j < 0) {
        best1[v] = KEY_NONE;
        best2[v] = 0xffffffffu;
        return;
    }
    const int mn = int(v) < j ? int(v) : j, mx = int(v) < j ? j : int(v);
    best1[v] = (uint64_t(__float_as_uint(dist[v * k])) << 32) | uint32_t(mn);
    best2[v] = unsigned(mx);
}

__global__ void bv_hook_kernel(const int32_t *__restrict__ comp, int64_t n,
                               const unsigned long long *__restrict__ best1,
                               const unsigned int *__restrict__ best2, int32_t *__restrict__ newp,
                               int32_t *__restrict__ flag, int32_t *__restrict__ rmn,
                               int32_t *__restrict__ rmx, float *__restrict__ rw) {
    int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= n) return;
    flag[c] = 0;
    if (comp[c] != c) return;  // not a component root
    unsigned long long b1 = best1[c];
    if (b1 == KEY_NONE) {
        newp[c] = int32_t(c);
        return;
    }
    int mn = int(uint32_t(b1));
    int mx = int(best2[c]);
    int cm = comp[mn], cx = comp[mx];
    int other = cm == int(c) ? cx : cm;
    bool mutual = best1[other] == b1 && best2[other] == unsigned(mx);
    if (mutual && c < other) {
        newp[c] = int32_t(c);
        return;
    }
    newp[c] = other;
    flag[c] = 1;
    rmn[c] = mn;
    rmx[c] = mx;
    rw[c] = __uint_as_float(uint32_t(b1 >> 32));
}

__global__ void bv_jump_kernel(const int32_t *__restrict__ comp, int64_t n, int32_t *newp_,
                               int limit, int *dstatus) {
    int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= n || comp[c] != c) return;
    volatile int32_t *newp = newp_;
    int guard = 0;
    while (guard++ < limit) {
        int p = newp[c];
        int g = newp[p];
        if (g == p) return;
        newp[c] = g;
    }
    set_status(dstatus, STATUS_LOOP_LIMIT);
}

__global__ void bv_relabel_kernel(int32_t *__restrict__ comp, int64_t n,
                                  const int32_t *__restrict__ newp) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = newp[comp[v]];
}

__global__ void bv_record_kernel(const int32_t *__restrict__ flag,
                                 const int32_t *__restrict__ pos, int64_t n, int64_t base,
                                 const int32_t *__restrict__ rmn, const int32_t *__restrict__ rmx,
                                 const float *__restrict__ rw, int32_t *__restrict__ tu,
                                 int32_t *__restrict__ tv, float *__restrict__ tw) {
    int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= n || !flag[c]) return;
    int64_t o = base + pos[c];
    if (o >= n - 1) return;  // a spanning tree has n-1 edges; never write past them
    tu[o] = rmn[c];
    tv[o] = rmx[c];
    tw[o] = rw[c];
}

// ------------------------------------------------------- FP64 weights

constexpr int WR_NT = 256;
constexpr int WR_IPT = 8;
constexpr int WR_TILE = WR_NT * WR_IPT;

// fixed-order block reduction of two double values per thread
__device__ void block_sum2(double &a, double &b) {
    __shared__ double sa[WR_NT], sb[WR_NT];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int s = WR_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    a = sa[0];
    b = sb[0];
}

template <int VEC>
__global__ void weight_partial_kernel(const float *__restrict__ X, int d,
                                      const int32_t *__restrict__ tu,
                                      const int32_t *__restrict__ tv,
                                      const float *__restrict__ tw, int64_t m,
                                      double *__restrict__ part) {
    int64_t base = int64_t(blockIdx.x) * WR_TILE + int64_t(threadIdx.x) * WR_IPT;
    double s32 = 0.0, s64 = 0.0;
    for (int r = 0; r < WR_IPT; ++r) {
        int64_t e = base + r;
        if (e >= m) break;
        s32 += double(tw[e]);
        if (X) {
            const float *a = X + int64_t(tu[e]) * d, *b = X + int64_t(tv[e]) * d;
            double p = 0.0;
            if constexpr (VEC == 4) {   // the same sum, 16-byte loads
                const float4 *a4 = reinterpret_cast<const float4 *>(a);
                const float4 *b4 = reinterpret_cast<const float4 *>(b);
                for (int q = 0; q < d / 4; ++q) {
                    const float4 x = __ldg(a4 + q), y = __ldg(b4 + q);
                    const double d0 = double(x.x) - double(y.x), d1 = double(x.y) - double(y.y);
                    const double d2 = double(x.z) - double(y.z), d3 = double(x.w) - double(y.w);
                    p = fma(d0, d0, p);
                    p = fma(d1, d1, p);
                    p = fma(d2, d2, p);
                    p = fma(d3, d3, p);
                }
            } else {
                for (int t = 0; t < d; ++t) {
                    double dl = double(a[t]) - double(b[t]);
                    p = fma(dl, dl, p);
                }
            }
            s64 += sqrt(p);
        }
    }
    block_sum2(s32, s64);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s32;
        part[2 * blockIdx.x + 1] = s64;
    }
}

__global__ void weight_final_kernel(const double *__restrict__ part, int64_t nb,
                                    double *__restrict__ W) {
    double s32 = 0.0, s64 = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += WR_NT) {
        s32 += part[2 * b];
        s64 += part[2 * b + 1];
    }
    block_sum2(s32, s64);
    if (threadIdx.x == 0) {
        W[0] = s32;
        W[1] = s64;
    }
}

// ----------------------------------------------------------- backward

template <int VEC>
__global__ void edge_len_kernel(const float *__restrict__ X, int d,
                                const int32_t *__restrict__ tu, const int32_t *__restrict__ tv,
                                int64_t m, float *__restrict__ wl) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < m) wl[e] = canon_dist<VEC>(X + int64_t(tu[e]) * d, X + int64_t(tv[e]) * d, d);
}

__global__ void incidence_kernel(const int32_t *__restrict__ tu, const int32_t *__restrict__ tv,
                                 int64_t m, uint32_t *__restrict__ keys, int32_t *__restrict__ vals,
                                 int32_t *__restrict__ deg) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    keys[2 * e] = uint32_t(tu[e]);
    vals[2 * e] = int32_t(2 * e);
    keys[2 * e + 1] = uint32_t(tv[e]);
    vals[2 * e + 1] = int32_t(2 * e + 1);
    atomicAdd(&deg[tu[e]], 1);
    atomicAdd(&deg[tv[e]], 1);
}

// gX[v][t] = gW * sum over v's edges, ascending edge index, of
// (x_v[t] - x_other[t]) / w_e  (w_e = 0 contributes 0)
__global__ void grad_kernel(const float *__restrict__ X, int64_t n, int d,
                            const int32_t *__restrict__ tu, const int32_t *__restrict__ tv,
                            const float *__restrict__ wl, const int32_t *__restrict__ off,
                            const int32_t *__restrict__ inc, float gW, float *__restrict__ gX) {
    int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * d) return;
    int64_t v = idx / d;
    int t = int(idx - v * d);
    float xs = X[idx];
    float acc = 0.0f;
    for (int q = off[v]; q < off[v + 1]; ++q) {
        int code = inc[q];
        int e = code >> 1;
        int other = (code & 1) ? tu[e] : tv[e];
        float w = wl[e];
        if (w > 0.0f) acc = __fadd_rn(acc, __fdiv_rn(__fsub_rn(xs, X[int64_t(other) * d + t]), w));
    }
    gX[idx] = __fmul_rn(gW, acc);
}

// Record the round's tree edges at base + pos (base and the round's count
// live on the device), then advance base and raise `done` when a round
// added no edge: the later rounds of a fixed budget become no-ops.
__global__ void bv_record_dev_kernel(const int32_t *__restrict__ flag,
                                     const int32_t *__restrict__ pos, int64_t n,
                                     const long long *__restrict__ base,
                                     const int32_t *__restrict__ rmn, const int32_t *__restrict__ rmx,
                                     const float *__restrict__ rw, int32_t *__restrict__ tu,
                                     int32_t *__restrict__ tv, float *__restrict__ tw,
                                     int64_t cap, const int *__restrict__ done) {
    if (*done) return;
    int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= n || !flag[c]) return;
    int64_t o = *base + pos[c];
    if (o >= cap) return;
    tu[o] = rmn[c];
    tv[o] = rmx[c];
    tw[o] = rw[c];
}

__global__ void bv_advance_kernel(long long *base, const int32_t *__restrict__ added, int *done,
                                  int *rounds) {
    if (*done) return;
    if (*added == 0) {
        *done = 1;
    } else {
        *base += *added;
        *rounds += 1;
    }
}

__global__ void bv_gate_kernel(const int *__restrict__ done, int32_t *__restrict__ flag, int64_t n) {
    // a finished forest records nothing more
    if (!*done) return;
    int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c < n) flag[c] = 0;
}

inline unsigned blocks_for(int64_t count, int th) { return unsigned((count + th - 1) / th); }

}  // namespace

size_t boruvka_workspace(int64_t n, int64_t ecap) {
    size_t b = align256(size_t(n) * 8) + align256(size_t(n) * 4) * 8 + scan_workspace(n) + 256;
    if (ecap > 0) b += align256(size_t(ecap) * 4) * 6 + 256;
    return b;
}

// Boruvka with no host synchronisation: a fixed budget of rounds, the
// edge count of E and the termination live on the device (for CUDA-graph
// capture). Finds the minimum spanning forest of the candidate graph.
famst_status boruvka_dev(const Exec &ex, Arena &ar, int64_t n, const int32_t *nbr,
                         const float *dist, int k, const int32_t *eu, const int32_t *ev,
                         const float *ew, int64_t m_cap, const int64_t *m_dev, MstOut out,
                         int64_t out_cap, int max_rounds, long long *edges_dev, int *rounds_dev) {
    if (n <= 1) return FAMST_OK;
    unsigned long long *best1 = ar.take<unsigned long long>(size_t(n));
    unsigned int *best2 = ar.take<unsigned int>(size_t(n));
    int32_t *comp = ar.take<int32_t>(size_t(n));
    int32_t *newp = ar.take<int32_t>(size_t(n));
    int32_t *flag = ar.take<int32_t>(size_t(n));
    int32_t *pos = ar.take<int32_t>(size_t(n));
    int32_t *rmn = ar.take<int32_t>(size_t(n));
    int32_t *rmx = ar.take<int32_t>(size_t(n));
    float *rw = ar.take<float>(size_t(n));
    int32_t *added = ar.take<int32_t>(1);
    int *done = ar.take<int>(1);
    if (!best1 || !best2 || !comp || !newp || !flag || !pos || !rmn || !rmx || !rw || !added ||
        !done)
        return FAMST_ERR_OOM;
    EdgeSrc es{nbr, dist, k, n * int64_t(k), eu, ev, ew, m_cap, m_dev};
    const int th = 256;
    int64_t nedges = es.nk + m_cap;
    unsigned egrid = blocks_for(nedges, th);
    unsigned ecap = unsigned(ex.num_sms) * 32;
    if (egrid > ecap) egrid = ecap;
    if (egrid == 0) egrid = 1;
    if (cudaMemsetAsync(done, 0, sizeof(int), ex.stream) != cudaSuccess ||
        cudaMemsetAsync(edges_dev, 0, sizeof(long long), ex.stream) != cudaSuccess ||
        cudaMemsetAsync(rounds_dev, 0, sizeof(int), ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, bv_init_kernel, blocks_for(n, th), th, 0, comp, n);
    for (int r = 0; r < max_rounds; ++r) {
        if (cudaMemsetAsync(best1, 0xff, size_t(n) * 8, ex.stream) != cudaSuccess ||
            cudaMemsetAsync(best2, 0xff, size_t(n) * 4, ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        FAMST_LAUNCH(ex, bv_min1_kernel, egrid, th, 0, es, comp, best1, done);
        FAMST_LAUNCH(ex, bv_min2_kernel, egrid, th, 0, es, comp, best1, best2, done);
        FAMST_LAUNCH(ex, bv_hook_kernel, blocks_for(n, th), th, 0, comp, n, best1, best2, newp,
                     flag, rmn, rmx, rw);
        FAMST_LAUNCH(ex, bv_gate_kernel, blocks_for(n, th), th, 0, done, flag, n);
        FAMST_LAUNCH(ex, bv_jump_kernel, blocks_for(n, th), th, 0, comp, n, newp,
                     ex.loop_limit > 0 ? ex.loop_limit : JUMP_LIMIT, ex.dstatus);
        FAMST_LAUNCH(ex, bv_relabel_kernel, blocks_for(n, th), th, 0, comp, n, newp);
        size_t mark = ar.off;
        famst_status st = exclusive_scan_i32(ex, ar, flag, pos, n, added);
        ar.off = mark;
        if (st != FAMST_OK) return st;
        FAMST_LAUNCH(ex, bv_record_dev_kernel, blocks_for(n, th), th, 0, flag, pos, n, edges_dev,
                     rmn, rmx, rw, out.tu, out.tv, out.tw, out_cap, done);
        FAMST_LAUNCH(ex, bv_advance_kernel, 1, 1, 0, edges_dev, added, done, rounds_dev);
    }
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

famst_status bv_state_init(const Exec &ex, Arena &ar, int64_t n, BvState *S, int64_t ecap) {
    S->n = n;
    if (ecap > 0) {
        S->ecap = ecap;
        for (int i = 0; i < 2; ++i) {
            S->cu[i] = ar.take<int32_t>(size_t(ecap));
            S->cv[i] = ar.take<int32_t>(size_t(ecap));
            S->cw[i] = ar.take<float>(size_t(ecap));
            if (!S->cu[i] || !S->cv[i] || !S->cw[i]) return FAMST_ERR_OOM;
        }
        S->ccount = ar.take<unsigned long long>(2);
        if (!S->ccount) return FAMST_ERR_OOM;
    }
    S->best1 = ar.take<unsigned long long>(size_t(n));
    S->best2 = ar.take<unsigned int>(size_t(n));
    S->comp = ar.take<int32_t>(size_t(n));
    S->newp = ar.take<int32_t>(size_t(n));
    S->flag = ar.take<int32_t>(size_t(n));
    S->pos = ar.take<int32_t>(size_t(n));
    S->rmn = ar.take<int32_t>(size_t(n));
    S->rmx = ar.take<int32_t>(size_t(n));
    S->rw = ar.take<float>(size_t(n));
    S->total = ar.take<int32_t>(1);
    if (!S->best1 || !S->best2 || !S->comp || !S->newp || !S->flag || !S->pos || !S->rmn ||
        !S->rmx || !S->rw || !S->total)
        return FAMST_ERR_OOM;
    FAMST_LAUNCH(ex, bv_init_kernel, blocks_for(n, 256), 256, 0, S->comp, n);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

// One Boruvka round over the kNN-style edges (i -> nbr[i*k + r]) plus
// (eu, ev): every component's minimum outgoing edge under (w, min, max)
// is hooked and recorded at out[base ...]; *added_host (pinned) receives
// the number of edges added. Synchronises.
famst_status bv_round(const Exec &ex, Arena &ar, BvState &S, const int32_t *nbr, const float *dist,
                      int k, const int32_t *eu, const int32_t *ev, const float *ew, int64_t m,
                      MstOut out, int64_t base, int32_t *added_host) {
    const int64_t n = S.n;
    EdgeSrc es{nbr, dist, k, n * int64_t(k), eu, ev, ew, m, nullptr};
    if (S.cur >= 0)   // the previous scan's edges between components
        es = EdgeSrc{nullptr, nullptr, 1, 0, S.cu[S.cur], S.cv[S.cur], S.cw[S.cur], S.ecap,
                      reinterpret_cast<const int64_t *>(S.ccount + S.cur)};
    const int th = 256;
    int64_t nedges = es.nk + es.m;
    unsigned egrid = blocks_for(nedges, th);
    unsigned ecap = unsigned(ex.num_sms) * 32;
    if (egrid > ecap) egrid = ecap;
    if (egrid == 0) egrid = 1;
    if (S.round == 0 && S.knn_exact && k >= 1) {
        FAMST_LAUNCH(ex, bv_first_kernel, blocks_for(n, th), th, 0, nbr, dist, k, n, S.best1,
                     S.best2);
    } else {
        if (cudaMemsetAsync(S.best1, 0xff, size_t(n) * 8, ex.stream) != cudaSuccess ||
            cudaMemsetAsync(S.best2, 0xff, size_t(n) * 4, ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        if (S.ecap > 0 && S.round >= 2) {   // early rounds keep most edges: no copy
            const int nxt = S.cur == 0 ? 1 : 0;
            if (cudaMemsetAsync(S.ccount + nxt, 0, 8, ex.stream) != cudaSuccess)
                return FAMST_ERR_CUDA;
            FAMST_LAUNCH(ex, bv_min1_kernel, egrid, th, 0, es, S.comp, S.best1, nullptr, S.cu[nxt],
                         S.cv[nxt], S.cw[nxt], S.ccount + nxt);
            FAMST_LAUNCH(ex, bv_min2_kernel, egrid, th, 0, es, S.comp, S.best1, S.best2, nullptr);
            S.cur = nxt;
        } else {
            FAMST_LAUNCH(ex, bv_min1_kernel, egrid, th, 0, es, S.comp, S.best1, nullptr, nullptr,
                         nullptr, nullptr, nullptr);
            FAMST_LAUNCH(ex, bv_min2_kernel, egrid, th, 0, es, S.comp, S.best1, S.best2, nullptr);
        }
    }
    ++S.round;
    FAMST_LAUNCH(ex, bv_hook_kernel, blocks_for(n, th), th, 0, S.comp, n, S.best1, S.best2, S.newp,
                 S.flag, S.rmn, S.rmx, S.rw);
    FAMST_LAUNCH(ex, bv_jump_kernel, blocks_for(n, th), th, 0, S.comp, n, S.newp,
                 ex.loop_limit > 0 ? ex.loop_limit : JUMP_LIMIT, ex.dstatus);
    FAMST_LAUNCH(ex, bv_relabel_kernel, blocks_for(n, th), th, 0, S.comp, n, S.newp);
    size_t mark = ar.off;  // the scan's scratch is reused by every round
    famst_status st = exclusive_scan_i32(ex, ar, S.flag, S.pos, n, S.total);
    ar.off = mark;
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, bv_record_kernel, blocks_for(n, th), th, 0, S.flag, S.pos, n, base, S.rmn,
                 S.rmx, S.rw, out.tu, out.tv, out.tw);
    if (cudaMemcpyAsync(added_host, S.total, 4, cudaMemcpyDeviceToHost, ex.stream) != cudaSuccess ||
        cudaStreamSynchronize(ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

famst_status boruvka(const Exec &ex, Arena &ar, int64_t n, const int32_t *nbr, const float *dist,
                     int k, const int32_t *eu, const int32_t *ev, const float *ew, int64_t m,
                     MstOut out, int64_t *tree_edges, int *rounds, int32_t *pinned_host,
                     bool knn_exact, bool compact) {
    *tree_edges = 0;
    *rounds = 0;
    if (n <= 1) return FAMST_OK;
    BvState S;
    famst_status st = bv_state_init(ex, ar, n, &S, compact ? n * int64_t(k) + m : 0);
    if (st != FAMST_OK) return st;
    S.knn_exact = knn_exact;
    int64_t got = 0;
    // at least half the components disappear every round that adds edges:
    // 64 rounds cover any n; the context's loop limit can lower the budget
    const int budget = ex.loop_limit > 0 && ex.loop_limit < 64 ? ex.loop_limit : 64;
    int32_t added = 0;
    for (int r = 0; r < budget && got < n - 1; ++r) {
        st = bv_round(ex, ar, S, nbr, dist, k, eu, ev, ew, m, out, got, pinned_host);
        if (st != FAMST_OK) return st;
        *rounds = r + 1;
        added = *pinned_host;
        if (added == 0) break;
        got += added;
    }
    *tree_edges = got;
    // the budget ran out while rounds still added edges: not a disconnected graph
    if (got < n - 1 && added > 0) return FAMST_ERR_TIMEOUT;
    return FAMST_OK;
}

size_t tree_weight_workspace(int64_t m) {
    return align256(size_t((m + WR_TILE - 1) / WR_TILE + 1) * 16);
}

famst_status tree_weight(const Exec &ex, Arena &ar, const float *X, int d, bool vec4,
                         const int32_t *tu, const int32_t *tv, const float *tw, int64_t m,
                         double *W_dev) {
    int64_t nb = (m + WR_TILE - 1) / WR_TILE;
    if (nb == 0) nb = 1;
    double *part = ar.take<double>(size_t(nb) * 2);
    if (!part) return FAMST_ERR_OOM;
    if (vec4)
        FAMST_LAUNCH(ex, weight_partial_kernel<4>, unsigned(nb), WR_NT, 0, X, d, tu, tv, tw, m,
                     part);
    else
        FAMST_LAUNCH(ex, weight_partial_kernel<1>, unsigned(nb), WR_NT, 0, X, d, tu, tv, tw, m,
                     part);
    FAMST_LAUNCH(ex, weight_final_kernel, 1, WR_NT, 0, part, nb, W_dev);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

size_t mst_backward_workspace(int64_t n, int64_t m) {
    return align256(size_t(m) * 4) + align256(size_t(2 * m) * 4) * 2 +
           align256(size_t(n + 1) * 4) * 2 + radix_sort_workspace(2 * m) + scan_workspace(n + 1);
}

famst_status mst_backward(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, bool vec4,
                          const int32_t *tu, const int32_t *tv, int64_t m, float gW, float *gX) {
    float *wl = ar.take<float>(size_t(m > 0 ? m : 1));
    uint32_t *keys = ar.take<uint32_t>(size_t(2 * m > 0 ? 2 * m : 1));
    int32_t *inc = ar.take<int32_t>(size_t(2 * m > 0 ? 2 * m : 1));
    int32_t *deg = ar.take<int32_t>(size_t(n + 1));
    int32_t *off = ar.take<int32_t>(size_t(n + 1));
    if (!wl || !keys || !inc || !deg || !off) return FAMST_ERR_OOM;
    const int th = 256;
    if (cudaMemsetAsync(deg, 0, size_t(n + 1) * 4, ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    if (m > 0) {
        if (vec4)
            FAMST_LAUNCH(ex, edge_len_kernel<4>, blocks_for(m, th), th, 0, X, d, tu, tv, m, wl);
        else
            FAMST_LAUNCH(ex, edge_len_kernel<1>, blocks_for(m, th), th, 0, X, d, tu, tv, m, wl);
        FAMST_LAUNCH(ex, incidence_kernel, blocks_for(m, th), th, 0, tu, tv, m, keys, inc, deg);
        int bits = 0;
        while ((int64_t(1) << bits) < n) ++bits;
        famst_status st = radix_sort_pairs(ex, ar, keys, inc, 2 * m, bits);
        if (st != FAMST_OK) return st;
    }
    famst_status st = exclusive_scan_i32(ex, ar, deg, off, n + 1, nullptr);
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, grad_kernel, blocks_for(n * d, th), th, 0, X, n, d, tu, tv, wl, off, inc, gW,
                 gX);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst
