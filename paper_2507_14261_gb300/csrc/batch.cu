// Many point clouds in one build (famst_build_batched).
//
// The clouds are independent FAMST builds. They are concatenated in a
// compact vertex space (cloud b = ids voff[b] .. voff[b+1]-1) with every row
// zero-padded to D columns; zero columns leave the canonical FP32 distance
// unchanged (fmaf(0, 0, p) = p), so each cloud's result is bit-identical to
// a build of that cloud alone. The kNN graph of the batch has no edge
// between clouds, so the graph phases run once over the whole batch:
//   Phase 1   tensor tiles over a padded row space in which every cloud
//             starts on a 256-row boundary (tiles never straddle clouds), or
//             FP32 tiles restricted to the cloud's keys -- chosen per cloud by
//             the autotuner below;
//   Alg. 2    one union-find over all ids; component indices are global, so
//             cloud b's components are cbase[b] .. cbase[b+1]-1 and the
//             cloud-local index is global - cbase[b];
//   Alg. 3    one launch over the pairs of all clouds (cloud b draws with
//             seed + b and cloud-local pair indices);
//   Alg. 4    one launch over all edges;
//   MST       Boruvka finds the minimum spanning forest (one tree per cloud)
//             with a fixed round budget and device-side termination;
// then the tree edges are grouped per cloud and summed in FP64 per cloud.
// Every count that depends on the data (components, pairs, edges) stays on
// the device, so the whole sequence is captured in a CUDA graph once and
// replayed; the host only reads the results after the replay.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "batch.cuh"

namespace famst {
namespace {

constexpr int STATUS_CAPACITY = 32;

__device__ __forceinline__ int cloud_of_v(const long long *__restrict__ off, int B, long long v) {
    int lo = 0, hi = B;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

// X_concat (cloud b: n_b rows of d_b floats) -> Xc (N rows of D floats, zero
// beyond d_b); flags NaN / Inf.
__global__ void bt_pack_kernel(const float *__restrict__ Xin, const long long *__restrict__ xoff,
                               const long long *__restrict__ voff, const int *__restrict__ dims,
                               int B, int64_t N, int D, float *__restrict__ Xc, int *dstatus) {
    int64_t v = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (v >= N) return;
    const int b = cloud_of_v(voff, B, v);
    const int d = dims[b];
    const float *src = Xin + xoff[b] + (v - voff[b]) * d;
    int bad = 0;
    for (int t = lane; t < D; t += 32) {
        float x = t < d ? src[t] : 0.0f;
        bad |= !isfinite(x);
        Xc[v * D + t] = x;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(dstatus, STATUS_NONFINITE);
}

// cbase[b] = global index of cloud b's first component (its first vertex is
// the smallest id of its component); cbase[B] = t.
__global__ void bt_cbase_kernel(const int32_t *__restrict__ comp, const long long *__restrict__ voff,
                                int B, const int32_t *__restrict__ t_dev, int32_t *__restrict__ cbase) {
    for (int b = threadIdx.x; b <= B; b += blockDim.x) cbase[b] = b < B ? comp[voff[b]] : *t_dev;
}

// pp[b] = pairs of the clouds before b; m = lambda * pp[B], capped.
__global__ void bt_pairs_kernel(const int32_t *__restrict__ cbase, int B, int lambda,
                                int64_t m_cap, long long *__restrict__ pp, int64_t *__restrict__ m_dev,
                                int64_t *__restrict__ m_req, int *dstatus) {
    if (threadIdx.x != 0) return;
    long long acc = 0;
    for (int b = 0; b < B; ++b) {
        pp[b] = acc;
        const long long t = cbase[b + 1] - cbase[b];
        acc += t * (t - 1) / 2;
    }
    pp[B] = acc;
    const int64_t m = int64_t(lambda) * acc;
    *m_req = m;
    *m_dev = m < m_cap ? m : m_cap;
    if (m > m_cap) set_status(dstatus, STATUS_CAPACITY);
}

__global__ void bt_iota_kernel(const int32_t *__restrict__ comp, int64_t n, uint32_t *__restrict__ keys,
                               int32_t *__restrict__ vals) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) {
        keys[v] = uint32_t(comp[v]);
        vals[v] = int32_t(v);
    }
}

__global__ void bt_segment_starts_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                         const int32_t *__restrict__ t_dev, int32_t *__restrict__ off) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n && (i == 0 || keys[i] != keys[i - 1])) off[keys[i]] = int32_t(i);
    if (i == 0) off[*t_dev] = int32_t(n);
}

__global__ void bt_tree_key_kernel(const int32_t *__restrict__ tu, int64_t m,
                                   const long long *__restrict__ voff, int B,
                                   uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    keys[e] = uint32_t(cloud_of_v(voff, B, tu[e]));
    vals[e] = int32_t(e);
}

// sorted by cloud (stable): position i holds cloud b's next tree edge in
// (round, component) order; write it with cloud-local ids
__global__ void bt_tree_gather_kernel(const uint32_t *__restrict__ keys, const int32_t *__restrict__ vals,
                                      int64_t m, const long long *__restrict__ voff,
                                      const int32_t *__restrict__ tu, const int32_t *__restrict__ tv,
                                      const float *__restrict__ tw, int32_t *__restrict__ ou,
                                      int32_t *__restrict__ ov, float *__restrict__ ow) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int b = int(keys[i]);
    const int e = vals[i];
    ou[i] = int32_t(tu[e] - voff[b]);
    ov[i] = int32_t(tv[e] - voff[b]);
    ow[i] = tw[e];
}

// one block per cloud: FP64 sum of its n_b - 1 tree weights in a fixed order
__global__ void bt_cloud_weight_kernel(const float *__restrict__ tw, const long long *__restrict__ voff,
                                       double *__restrict__ W) {
    __shared__ double red[256];
    const int b = blockIdx.x;
    const long long e0 = voff[b] - b, e1 = voff[b + 1] - b - 1;
    double s = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += double(tw[e]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) W[b] = red[0];
}

__global__ void bt_check_forest_kernel(const long long *__restrict__ edges, int64_t want, int *dstatus) {
    if (*edges != want) set_status(dstatus, STATUS_DISCONNECTED);
}

// Spatial order of the tensor clouds' rows (their key tiles are then visited
// outward from the query tile's own, so the candidate lists meet near keys
// first): sort key of row v = its cloud in the top cb bits, then the top
// bits of its projection on a fixed +-1 direction (order-preserving bits of
// the FP32 value). Rows of FP32-tile clouds keep their order (projection
// bits 0; the sort is stable).
__global__ void bt_proj_key_kernel(const float *__restrict__ Xc, int D, int64_t N,
                                   const long long *__restrict__ voff, int B,
                                   const CloudDev *__restrict__ cl, int cb,
                                   uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    const int64_t v = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= N) return;
    const int b = cloud_of_v(voff, B, v);
    const bool tc = cl[b].use_tc != 0;
    float p = 0.0f;
    if (tc)
        for (int t = lane; t < D; t += 32) {
            const float x = Xc[v * D + t];
            p += ((uint32_t(t) * 0x9E3779B1u) >> 31) ? x : -x;
        }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0) {
        uint32_t u = __float_as_uint(p);
        u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        const uint32_t hi = cb > 0 ? uint32_t(b) << (32 - cb) : 0u;
        const uint32_t lo = tc ? (cb > 0 ? u >> cb : u) : 0u;
        keys[v] = hi | lo;
        vals[v] = int32_t(v);
    }
}

__global__ void bt_gather_rows_kernel(const float *__restrict__ Xc, int D, int64_t N,
                                      const int32_t *__restrict__ perm, float *__restrict__ Xs) {
    const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const float *src = Xc + int64_t(perm[i]) * D;
    for (int t = lane; t < D; t += 32) Xs[i * D + t] = src[t];
}

// deterministic pseudo-random fill (SplitMix-style hash), for timing runs
__global__ void bt_fill_kernel(float *p, int64_t count, uint32_t salt) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint64_t z = uint64_t(i) * 0x9E3779B97F4A7C15ull + salt;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    p[i] = float(z >> 40) * (1.0f / 16777216.0f);
}

inline unsigned blocks_for(int64_t count, int th) { return unsigned((count + th - 1) / th); }
inline int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------- autotuner
//
// For each class of clouds (K extent of the tensor tiles, d, n rounded up to
// a power of two, k, precision) it times
// the exact kNN of a synthetic cloud of that class on both paths and keeps
// the faster one. Results are cached per process and, when the environment
// variable FAMST_AUTOTUNE_CACHE names a file, appended to / read from it.
using TuneKey = std::tuple<int, int, int, int, int, int>;  // device, d_pad, d, log2 n, k, x3
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;  // 1 = tensor tiles, 0 = FP32 tiles
bool g_tune_loaded = false;

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("FAMST_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    int a, b, c, d, e, g, h;
    while (std::fscanf(f, "%d %d %d %d %d %d %d", &a, &b, &c, &d, &e, &g, &h) == 7)
        g_tune[TuneKey(a, b, c, d, e, g)] = h;
    std::fclose(f);
}

void tune_store(const TuneKey &key, int choice) {
    const char *path = std::getenv("FAMST_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %d %d %d %d %d\n", std::get<0>(key), std::get<1>(key), std::get<2>(key),
                 std::get<3>(key), std::get<4>(key), std::get<5>(key), choice);
    std::fclose(f);
}

double time_ms(const Exec &ex, const std::function<famst_status()> &fn, famst_status *st) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    *st = fn();  // warm-up
    cudaEventRecord(a, ex.stream);
    if (*st == FAMST_OK) *st = fn();
    cudaEventRecord(b, ex.stream);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

int batch_autotune(const Exec &ex, int d, int64_t n, int k, bool x3) {
    const int d_pad = int(up(d, 64));
    int lg = 9;
    while ((int64_t(1) << lg) < n && lg < 15) ++lg;
    int dev = 0;
    cudaGetDevice(&dev);
    const TuneKey key(dev, d_pad, d, lg, k, int(x3));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    int choice = 0;
    if (knn_tc_supported(int64_t(1) << lg, d, k, x3)) {
        const int64_t nn = int64_t(1) << lg;
        const size_t ws = knn_tc_workspace(nn, d, k, x3, ex.num_sms) +
                          knn_fp32_workspace(nn, d, k, nn, ex.num_sms) + (size_t(1) << 20);
        char *buf = nullptr;
        float *X = nullptr;
        int32_t *nbr = nullptr;
        float *dist = nullptr;
        int32_t *pinned = nullptr;
        if (cudaMalloc(&buf, ws) == cudaSuccess && cudaMalloc(&X, size_t(nn) * d * 4) == cudaSuccess &&
            cudaMalloc(&nbr, size_t(nn) * k * 4) == cudaSuccess &&
            cudaMalloc(&dist, size_t(nn) * k * 4) == cudaSuccess &&
            cudaMallocHost(&pinned, 64) == cudaSuccess) {
            bt_fill_kernel<<<blocks_for(nn * d, 256), 256, 0, ex.stream>>>(X, nn * d, 12345u);
            const bool v4 = (d % 4 == 0);
            famst_status s1, s2;
            double t_tc = time_ms(ex, [&]() {
                Arena ar{buf, ws, 0};
                int64_t unc = 0;
                return knn_tc(ex, ar, X, nn, d, k, x3, v4, nbr, dist, pinned, &unc);
            }, &s1);
            double t_f32 = time_ms(ex, [&]() {
                Arena ar{buf, ws, 0};
                return knn_fp32(ex, ar, X, nn, d, k, nullptr, 0, nn, nbr, dist);
            }, &s2);
            if (s1 == FAMST_OK && s2 == FAMST_OK) choice = t_tc < t_f32 ? 1 : 0;
        }
        cudaGetLastError();
        if (buf) cudaFree(buf);
        if (X) cudaFree(X);
        if (nbr) cudaFree(nbr);
        if (dist) cudaFree(dist);
        if (pinned) cudaFreeHost(pinned);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = choice;
    tune_store(key, choice);
    return choice;
}

// Tile shapes of the batched tensor pass (epilogue warps and ring stages),
// timed on the batch's own prepared operands; the pick is cached per
// (device, operand width, k, precision, log2 of the work items).
using ShapeKey = std::tuple<int, int, int, int, int>;
std::map<ShapeKey, int> g_shape;   // guarded by g_tune_mu

famst_status batch_tune_tiles(const Exec &ex, BatchPlan &P) {
    if (!P.any_tc || P.n_shapes < 2) return FAMST_OK;
    const int64_t items = int64_t(P.tct.size());
    int lg = 0;
    while ((int64_t(1) << lg) < items) ++lg;
    int dev = 0;
    cudaGetDevice(&dev);
    const ShapeKey key(dev, P.D, P.k, int(P.x3), lg);
    int pick = -1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_shape.find(key);
        if (it != g_shape.end()) pick = it->second;
    }
    if (pick < 0) {
        double best = 0.0;
        for (int sh = 0; sh < P.n_shapes; ++sh) {
            famst_status st = FAMST_OK;
            const double ms = time_ms(ex, [&]() {
                return knn_tc_batched_tiles(ex, P.D, P.x3, P.shape_stages[sh], P.shape_smem[sh],
                                            P.tc_kc, P.shape_epi[sh], P.dev.tct, items, P.dev.ny,
                                            P.dev.cand, P.dev.splus, &P.mA, &P.mB, true);
            }, &st);
            if (st != FAMST_OK) return st;
            if (pick < 0 || ms < best) {
                best = ms;
                pick = sh;
            }
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_shape[key] = pick;
    }
    P.tc_epi = P.shape_epi[pick];
    P.tc_stages = P.shape_stages[pick];
    P.tc_smem = P.shape_smem[pick];
    return FAMST_OK;
}

// ------------------------------------------------------------------ plan

famst_status batch_plan(const Exec &ex, const int64_t *offsets, const int32_t *dims, int B, int k,
                        int lambda, int prec, int max_iters, int64_t m_cap, BatchPlan *P) {
    P->B = B;
    P->k = k;
    P->lambda = lambda;
    P->prec = prec;
    P->max_iters = max_iters;
    P->x3 = prec == FAMST_PREC_BF16X3;
    P->voff.assign(B + 1, 0);
    P->roff.assign(B + 1, 0);
    P->xoff.assign(B + 1, 0);
    P->dims.assign(dims, dims + B);
    int dmax = 1, nmax = 2;
    for (int b = 0; b < B; ++b) {
        const int64_t nb = offsets[b + 1] - offsets[b];
        P->voff[b + 1] = P->voff[b] + nb;
        P->roff[b + 1] = P->roff[b] + up(nb, 256);
        P->xoff[b + 1] = P->xoff[b] + nb * dims[b];
        dmax = std::max(dmax, int(dims[b]));
        nmax = std::max<int>(nmax, int(nb));
    }
    P->N = P->voff[B];
    P->NP = P->roff[B];
    P->D = int(up(dmax, 64));
    P->cl.resize(B);
    P->tct.clear();
    P->f32t.clear();
    bool any_tc = false;
    int tc_stages = 0, tc_kc = 32, tc_epi = 4;
    size_t tc_smem = 0;
    const bool tc_ok = prec != FAMST_PREC_FP32 &&
                       knn_tc_batched_plan(P->D, k, P->x3, 4, &tc_stages, &tc_smem, &tc_kc, &tc_epi);
    P->n_shapes = 0;
    if (tc_ok) {
        P->shape_epi[0] = tc_epi;
        P->shape_stages[0] = tc_stages;
        P->shape_smem[0] = tc_smem;
        P->n_shapes = 1;
        int s8 = 0, kc8 = 0, e8 = 0;
        size_t m8 = 0;
        if (knn_tc_batched_plan(P->D, k, P->x3, 8, &s8, &m8, &kc8, &e8) && e8 == 8 &&
            kc8 == tc_kc) {
            P->shape_epi[1] = 8;
            P->shape_stages[1] = s8;
            P->shape_smem[1] = m8;
            P->n_shapes = 2;
        }
    }
    for (int b = 0; b < B; ++b) {
        const int nb = int(P->voff[b + 1] - P->voff[b]);
        CloudDev &c = P->cl[b];
        c.voff = P->voff[b];
        c.n = nb;
        c.d = dims[b];
        c.d_pad = int(up(dims[b], 64));
        c.use_tc = (tc_ok && batch_autotune(ex, dims[b], nb, k, P->x3)) ? 1 : 0;
        if (c.use_tc) {
            any_tc = true;
            const int kt0 = int(P->roff[b] / 256), kt1 = kt0 + int(up(nb, 256) / 256);
            for (int q = 0; q < nb; q += 128)
                P->tct.push_back(TcTile{int(P->roff[b]) + q, kt0, kt1, c.d_pad / 64,
                                        int(P->roff[b]) + nb, int(P->roff[b] - P->voff[b])});
        } else {
            const int nt = int(up(nb, 128) / 128);
            for (int q = 0; q < nb; q += 64)
                P->f32t.push_back(F32Tile{int(P->voff[b]) + q, std::min(64, nb - q), 0, nt,
                                          int(P->voff[b]), int(P->voff[b]) + nb, dims[b], 0});
        }
    }
    P->any_tc = any_tc;
    P->tc_stages = tc_stages;
    P->tc_smem = tc_smem;
    P->tc_kc = tc_kc;
    P->tc_epi = tc_epi;
    int rounds = 2;
    while ((1 << (rounds - 2)) < nmax) ++rounds;
    P->max_rounds = rounds + 2;
    P->m_cap = m_cap;
    P->tree_m = P->N - B;
    return FAMST_OK;
}

size_t batch_workspace(const BatchPlan &P) {
    const int64_t N = P.N, NP = P.NP, D = P.D, B = P.B, k = P.k, m = P.m_cap;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += align256(bytes); };
    add(size_t(B + 1) * 8 * 3);                  // voff, roff, xoff
    add(size_t(B) * 4);                          // dims
    add(size_t(B) * sizeof(CloudDev));
    add(P.tct.size() * sizeof(TcTile) + 16);
    add(P.f32t.size() * sizeof(F32Tile) + 16);
    add(size_t(N) * D * 4);                      // Xc
    add(size_t(N) * k * 4 * 2);                  // nbr, dist
    if (P.any_tc) {
        add(size_t(NP) * (P.x3 ? 2 : 1) * D * 2);  // H
        add(size_t(NP) * 4);                       // ny
        add(size_t(N) * 4);                        // xn2
        add(size_t(B) * D * 4);                    // means
        add(size_t(B) * 4);                        // ymax
        add(size_t(N) * (P.tc_kc - 1) * 4);        // candidates
        add(size_t(N) * 4 * 2 + 256);              // splus, fail rows, count
        add(size_t(N) * D * 4);                    // rows in spatial order
        add(size_t(N) * 4);                        // their permutation
    }
    if (!P.f32t.empty())
        add(size_t(N) * (P.k + 8) * 8 + size_t(N) * 4 + 512);  // FP32 candidates, fails
    add(size_t(N) * 4 * 3);                      // comp, members, keys
    add(size_t(N + 1) * 4);                      // comp_off
    add(size_t(B + 1) * 4 + size_t(B + 1) * 8 + 256);  // cbase, pp, counters
    add(size_t(m > 0 ? m : 1) * 4 * 5);          // E
    add(size_t(N + 1) * 4 + size_t(N) * k * 4);  // reverse CSR
    add(size_t(P.max_iters + 1) * 4);            // refine histogram
    add(size_t(N) * 12 + 256);                   // forest (global ids)
    add(size_t(N) * 4 * 2);                      // tree keys / order
    add(size_t(B) * 8);                          // W
    add(size_t(P.xoff.back()) * 4);              // copy of the clouds
    add(size_t(N) * 12);                         // trees before the copy out
    b += components_workspace(N) + radix_sort_workspace(N) + reverse_csr_workspace(N, int(k)) +
         boruvka_workspace(N) + 8 * 4096;
    return b;
}

famst_status batch_bind(BatchPlan &P, char *base, size_t cap, cudaStream_t s) {
    Arena ar{base, cap, 0};
    const int B = P.B;
    const int64_t N = P.N, NP = P.NP, D = P.D, k = P.k;
    const int64_t m = P.m_cap > 0 ? P.m_cap : 1;
    BatchDev &V = P.dev;
    V.voff = ar.take<long long>(B + 1);
    V.roff = ar.take<long long>(B + 1);
    V.xoff = ar.take<long long>(B + 1);
    V.dims = ar.take<int>(B);
    V.cl = ar.take<CloudDev>(B);
    V.tct = ar.take<TcTile>(P.tct.size() + 1);
    V.f32t = ar.take<F32Tile>(P.f32t.size() + 1);
    V.Xc = ar.take<float>(size_t(N) * D);
    V.nbr = ar.take<int32_t>(size_t(N) * k);
    V.dist = ar.take<float>(size_t(N) * k);
    if (P.any_tc) {
        V.H = ar.take<__nv_bfloat16>(size_t(NP) * (P.x3 ? 2 : 1) * D);
        V.ny = ar.take<float>(size_t(NP));
        V.xn2 = ar.take<float>(size_t(N));
        V.mean = ar.take<float>(size_t(B) * D);
        V.ymax = ar.take<unsigned>(B);
        V.cand = ar.take<int32_t>(size_t(N) * (P.tc_kc - 1));
        V.splus = ar.take<float>(size_t(N));
        V.fail_rows = ar.take<int32_t>(size_t(N));
        V.fail_count = ar.take<int32_t>(1);
        V.Xs = ar.take<float>(size_t(N) * D);
        V.perm = ar.take<int32_t>(size_t(N));
        if (!V.H || !V.ny || !V.xn2 || !V.mean || !V.ymax || !V.cand || !V.splus || !V.fail_rows ||
            !V.fail_count || !V.Xs || !V.perm)
            return FAMST_ERR_OOM;
        if (!knn_tc_batched_maps(V.H, NP, int(D), P.x3, &P.mA, &P.mB)) return FAMST_ERR_CUDA;
    }
    if (!P.f32t.empty()) {
        const int64_t kp = k + 8;
        V.f32c = ar.take<int32_t>(size_t(N) * kp);
        V.f32w = ar.take<float>(size_t(N) * kp);
        V.f32fail = ar.take<int32_t>(size_t(N));
        V.f32nfail = ar.take<int32_t>(1);
        if (!V.f32c || !V.f32w || !V.f32fail || !V.f32nfail) return FAMST_ERR_OOM;
    }
    V.comp = ar.take<int32_t>(size_t(N));
    V.members = ar.take<int32_t>(size_t(N));
    V.keys = ar.take<uint32_t>(size_t(N));
    V.comp_off = ar.take<int32_t>(size_t(N + 1));
    V.cbase = ar.take<int32_t>(B + 1);
    V.pp = ar.take<long long>(B + 1);
    V.t_dev = ar.take<int32_t>(1);
    V.m_dev = ar.take<int64_t>(1);
    V.m_req = ar.take<int64_t>(1);
    V.tree_edges = ar.take<long long>(1);
    V.rounds = ar.take<int>(1);
    V.eu = ar.take<int32_t>(m);
    V.ev = ar.take<int32_t>(m);
    V.ew = ar.take<float>(m);
    V.eci = ar.take<int32_t>(m);
    V.ecj = ar.take<int32_t>(m);
    V.rev_off = ar.take<int32_t>(size_t(N + 1));
    V.rev_src = ar.take<int32_t>(size_t(N) * k);
    V.hist = ar.take<int32_t>(size_t(P.max_iters + 1));
    V.fu = ar.take<int32_t>(size_t(N));
    V.fv = ar.take<int32_t>(size_t(N));
    V.fw = ar.take<float>(size_t(N));
    V.tkeys = ar.take<uint32_t>(size_t(N));
    V.tvals = ar.take<int32_t>(size_t(N));
    V.W = ar.take<double>(B);
    V.Xin = ar.take<float>(size_t(P.xoff.back() > 0 ? P.xoff.back() : 1));
    V.out_u = ar.take<int32_t>(size_t(N));
    V.out_v = ar.take<int32_t>(size_t(N));
    V.out_w = ar.take<float>(size_t(N));
    if (!V.voff || !V.roff || !V.xoff || !V.dims || !V.cl || !V.tct || !V.f32t || !V.Xc || !V.nbr ||
        !V.dist || !V.comp || !V.members || !V.keys || !V.comp_off || !V.cbase || !V.pp ||
        !V.t_dev || !V.m_dev || !V.m_req || !V.tree_edges || !V.rounds || !V.eu || !V.ev || !V.ew ||
        !V.eci || !V.ecj || !V.rev_off || !V.rev_src || !V.hist || !V.fu || !V.fv || !V.fw ||
        !V.tkeys || !V.tvals || !V.W || !V.Xin || !V.out_u || !V.out_v || !V.out_w)
        return FAMST_ERR_OOM;
    P.scratch_off = ar.off;
    // tables (synchronous copies: this runs before any capture)
    auto up_ = [&](void *dst, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    bool ok = up_(V.voff, P.voff.data(), size_t(B + 1) * 8) && up_(V.roff, P.roff.data(), size_t(B + 1) * 8) &&
              up_(V.xoff, P.xoff.data(), size_t(B + 1) * 8) && up_(V.dims, P.dims.data(), size_t(B) * 4) &&
              up_(V.cl, P.cl.data(), size_t(B) * sizeof(CloudDev)) &&
              up_(V.tct, P.tct.data(), P.tct.size() * sizeof(TcTile)) &&
              up_(V.f32t, P.f32t.data(), P.f32t.size() * sizeof(F32Tile));
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) return FAMST_ERR_CUDA;
    return FAMST_OK;
}

// ------------------------------------------------------------- enqueue

famst_status batch_enqueue(const Exec &ex, BatchPlan &P, char *base, size_t cap, uint64_t seed,
                           BatchHost *host) {
    BatchDev &V = P.dev;
    const float *X = V.Xin;
    int32_t *tu = V.out_u, *tv = V.out_v;
    float *tw = V.out_w;
    Arena ar{base, cap, P.scratch_off};
    const int B = P.B, k = P.k;
    const int64_t N = P.N, D = P.D;
    const int th = 256;
#define ST_(x)                                     \
    do {                                           \
        famst_status s_ = (x);                     \
        if (s_ != FAMST_OK) return s_;             \
    } while (0)
    if (cudaMemsetAsync(ex.dstatus, 0, sizeof(int), ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, bt_pack_kernel, blocks_for(N * 32, th), th, 0, X, V.xoff, V.voff, V.dims, B, N,
                 int(D), V.Xc, ex.dstatus);
    // Phase 1
    if (P.any_tc) {
        // the tensor clouds' rows in a spatial order (V.keys is free until Alg. 2)
        int cb = 0;
        while ((int64_t(1) << cb) < B) ++cb;
        FAMST_LAUNCH(ex, bt_proj_key_kernel, blocks_for(N * 32, th), th, 0, V.Xc, int(D), N,
                     V.voff, B, V.cl, cb, V.keys, V.perm);
        {
            size_t mark = ar.off;
            ST_(radix_sort_pairs(ex, ar, V.keys, V.perm, N, 32));
            ar.off = mark;
        }
        FAMST_LAUNCH(ex, bt_gather_rows_kernel, blocks_for(N * 32, th), th, 0, V.Xc, int(D), N,
                     V.perm, V.Xs);
        ST_(knn_tc_batched(ex, V.Xs, int(D), N, P.NP, V.voff, V.roff, B, V.cl, V.tct,
                           int64_t(P.tct.size()), k, P.x3, P.tc_stages, P.tc_smem, P.tc_kc,
                           P.tc_epi, V.H,
                           V.ny, V.xn2, V.mean, V.ymax, V.cand, V.splus, V.fail_rows, V.fail_count,
                           V.nbr, V.dist, &P.mA, &P.mB, V.Xc, V.perm));
    }
    if (!P.f32t.empty())
        ST_(knn_fp32_batched(ex, V.Xc, int(D), V.voff, B, V.cl, k, k + 8, V.f32t,
                             int64_t(P.f32t.size()), V.f32c, V.f32w, V.f32fail, V.f32nfail, V.nbr,
                             V.dist));
    // Alg. 2
    ST_(components_uf(ex, ar, V.nbr, N, k, V.comp, V.t_dev));
    FAMST_LAUNCH(ex, bt_cbase_kernel, 1, 256, 0, V.comp, V.voff, B, V.t_dev, V.cbase);
    FAMST_LAUNCH(ex, bt_pairs_kernel, 1, 32, 0, V.cbase, B, P.lambda, P.m_cap, V.pp, V.m_dev,
                 V.m_req, ex.dstatus);
    FAMST_LAUNCH(ex, bt_iota_kernel, blocks_for(N, th), th, 0, V.comp, N, V.keys, V.members);
    int bits = 0;
    while ((int64_t(1) << bits) < N) ++bits;
    {
        size_t mark = ar.off;
        ST_(radix_sort_pairs(ex, ar, V.keys, V.members, N, bits));
        ar.off = mark;
    }
    FAMST_LAUNCH(ex, bt_segment_starts_kernel, blocks_for(N, th), th, 0, V.keys, N, V.t_dev,
                 V.comp_off);
    // Alg. 3
    if (P.m_cap > 0)
        ST_(connect_edges_batched(ex, V.Xc, int(D), int(D), V.members, V.comp_off, V.pp, V.cbase, B,
                                  P.lambda, seed, P.m_cap, V.eu, V.ev, V.ew, V.eci, V.ecj));
    // Alg. 4
    {
        size_t mark = ar.off;
        ST_(reverse_csr(ex, ar, V.nbr, N, k, V.rev_off, V.rev_src));
        ar.off = mark;
    }
    if (cudaMemsetAsync(V.hist, 0, size_t(P.max_iters + 1) * 4, ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    if (P.m_cap > 0) {
        size_t mark = ar.off;
        ST_(refine_edges_dev(ex, ar, V.Xc, int(D), true, V.nbr, k, V.rev_off, V.rev_src, V.comp,
                             V.eu, V.ev, V.ew, V.eci, V.ecj, P.m_cap, V.m_dev, P.max_iters, V.hist));
        ar.off = mark;
    }
    // MST: spanning forest, then per cloud
    {
        size_t mark = ar.off;
        ST_(boruvka_dev(ex, ar, N, V.nbr, V.dist, k, V.eu, V.ev, V.ew, P.m_cap, V.m_dev,
                        MstOut{V.fu, V.fv, V.fw}, P.tree_m, P.max_rounds, V.tree_edges, V.rounds));
        ar.off = mark;
    }
    FAMST_LAUNCH(ex, bt_check_forest_kernel, 1, 1, 0, V.tree_edges, P.tree_m, ex.dstatus);
    if (P.tree_m > 0) {
        FAMST_LAUNCH(ex, bt_tree_key_kernel, blocks_for(P.tree_m, th), th, 0, V.fu, P.tree_m, V.voff,
                     B, V.tkeys, V.tvals);
        int cbits = 0;
        while ((1 << cbits) < B) ++cbits;
        size_t mark = ar.off;
        ST_(radix_sort_pairs(ex, ar, V.tkeys, V.tvals, P.tree_m, cbits));
        ar.off = mark;
        FAMST_LAUNCH(ex, bt_tree_gather_kernel, blocks_for(P.tree_m, th), th, 0, V.tkeys, V.tvals,
                     P.tree_m, V.voff, V.fu, V.fv, V.fw, tu, tv, tw);
    }
    FAMST_LAUNCH(ex, bt_cloud_weight_kernel, B, 256, 0, tw, V.voff, V.W);
    // results to pinned host memory (part of the same sequence)
    bool ok = cudaMemcpyAsync(host->W, V.W, size_t(B) * 8, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess &&
              cudaMemcpyAsync(host->cbase, V.cbase, size_t(B + 1) * 4, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess &&
              cudaMemcpyAsync(host->hist, V.hist, size_t(P.max_iters + 1) * 4, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess &&
              cudaMemcpyAsync(&host->words[0], V.m_req, 8, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess &&
              cudaMemcpyAsync(&host->words[1], V.tree_edges, 8, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess &&
              cudaMemcpyAsync(&host->words[2], V.rounds, 4, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess &&
              cudaMemcpyAsync(&host->words[3], ex.dstatus, 4, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess &&
              (!P.any_tc || cudaMemcpyAsync(&host->words[4], V.fail_count, 4, cudaMemcpyDeviceToHost, ex.stream) == cudaSuccess);
#undef ST_
    if (!ok) return FAMST_ERR_CUDA;
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

int batch_status_capacity() { return STATUS_CAPACITY; }

}  // namespace famst
