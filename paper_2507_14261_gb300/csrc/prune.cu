// Tile pruning for Phase 1 (exact kNN). Brute force visits every (query
// tile, key tile) pair; on data with structure most pairs cannot hold a
// neighbour, and the triangle inequality proves it cheaply:
//
//   1. Locality partition. Pivots: evenly spaced rows, then two coverage
//      passes that add pivots among the points far from every pivot (a
//      cluster without a pivot would otherwise scatter into foreign cells).
//      Every point joins the cell of its nearest pivot (the tensor-core
//      distance tiles with pivots as keys, BF16, top-1 -- any assignment is
//      valid, a good one only makes cells tight). Cells are ordered along the
//      pivots' minimum spanning tree, group by group (single linkage), and
//      points sorted by cell, so a 128-row query tile or a 256-row key tile
//      of the sorted order covers a few neighbouring cells (a tile with more
//      than NPMAX cells gets one ball of its own).
//   2. Balls. R_c >= max over members of |x - p_c| and D_lo(a, b) <=
//      |p_a - p_b| (warp-wide fast sums with rigorous rounding bounds).
//      For x in cell a and y in cell b: |x - y| >= D_lo(a, b) - R_a - R_b.
//   3. Radius of interest. For every point, any k other points give an
//      upper bound on its k-th neighbour distance: tau_r = the largest
//      distance (rounded up) to k points next to it in the sorted order,
//      inside its cell when the cell is large enough. tau_Q = max over the
//      query tile.
//   4. Lists. Key tile T is visited by query tile Q unless
//      LB(Q, T) = min over cells a of Q, b of T of D_lo - R_a - R_b exceeds
//      tau_Q (with a margin for the canonical rounding). skip_Q = the
//      smallest LB of the skipped tiles: every skipped key is at true
//      distance >= skip_Q from every point of Q.
//
// The re-rank certificate then also requires skip (1 - eps_canon) to exceed
// the k-th canonical distance; rows that fail fall back to the exact FP32
// tiles, so the output is the exact kNN whatever the data.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "famst_internal.cuh"

namespace famst {
namespace {

constexpr int QT = 128;    // query tile rows
constexpr int KT = 256;    // key tile rows
constexpr int NPMAX = 8;   // cells per tile beyond which a tile uses one enclosing ball

inline unsigned nblk(int64_t n, int th) { return unsigned((n + th - 1) / th); }

__device__ __forceinline__ float sq_hi(float p, float rho) {
    return __fadd_ru(__fmul_ru(p, 1.0f + rho), 1e-30f);
}
__device__ __forceinline__ float sq_lo(float p, float rho) {
    return fmaxf(__fsub_rd(__fmul_rd(p, 1.0f - rho), 1e-30f), 0.0f);
}

// pivot c = rows[c] (null: row c n / K): its operand row and norm; nyp
// padded with +inf up to Kpad
__global__ void pivots_kernel(const __nv_bfloat16 *__restrict__ H, int kh,
                              const float *__restrict__ ny, int64_t n, int K, int Kpad,
                              const int32_t *__restrict__ rows, int32_t *__restrict__ piv,
                              __nv_bfloat16 *__restrict__ Hp, float *__restrict__ nyp) {
    const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= Kpad) return;
    if (c >= K) {
        if (lane == 0) nyp[c] = __int_as_float(0x7f800000);
        return;
    }
    const int64_t row = rows ? int64_t(rows[c]) : c * n / K;
    if (lane == 0) {
        piv[c] = int32_t(row);
        nyp[c] = ny[row];
    }
    const uint4 *src = reinterpret_cast<const uint4 *>(H + row * kh);
    uint4 *dst = reinterpret_cast<uint4 *>(Hp + c * kh);
    for (int q = lane; q < kh / 8; q += 32) dst[q] = src[q];
}

// sort key of the points farthest from their pivot first: the approximate
// squared distance ||x'||^2 + s of the top-1 score s, descending
__global__ void far_key_kernel(const float *__restrict__ xn2, const float *__restrict__ s,
                               int64_t n, uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float d2 = fmaxf(xn2[i] + s[i], 0.0f);
    keys[i] = ~__float_as_uint(d2 == d2 ? d2 : 0.0f);
    vals[i] = int32_t(i);
}

// Picks among the points sorted by distance to their pivot, farthest first:
// F = how many lie beyond twice the median distance (4x in squared terms);
// pick j takes sorted entry floor(j F / Me), so the picks spread evenly over
// the far points instead of piling into the few most isolated groups.
__global__ void far_pick_kernel(const uint32_t *__restrict__ keys, const int32_t *__restrict__ vals,
                                int64_t n, int M, int32_t *__restrict__ rows,
                                int32_t *__restrict__ me_out) {
    __shared__ long long F_s;
    if (threadIdx.x == 0) {
        const float med = __uint_as_float(~keys[n / 2]);
        const float thr = 4.0f * med;
        // keys ascend = distances descend: first index with distance <= thr
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (__uint_as_float(~keys[mid]) > thr) lo = mid + 1; else hi = mid;
        }
        F_s = lo;
    }
    __syncthreads();
    // about one new pivot per 32 far points; the remaining slots repeat the
    // point nearest its pivot (a pivot itself), which adds no cell
    const int64_t F = F_s;
    const int64_t Me = F / 32 < M ? F / 32 : M;
    if (threadIdx.x == 0) *me_out = int32_t(Me);
    for (int j = threadIdx.x; j < M; j += blockDim.x)
        rows[j] = j < Me ? vals[int64_t(j) * F / Me] : vals[n - 1];
}

// cell of every point = the rank of its best pivot candidate; sort keys and
// cell sizes
__global__ void assign_kernel(const int32_t *__restrict__ cand, int kp, int64_t n, int K,
                              const int32_t *__restrict__ rank, uint32_t *__restrict__ keys,
                              int32_t *__restrict__ vals, int32_t *__restrict__ ccount) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cand[i * kp];
    if (c < 0 || c >= K) c = 0;
    c = rank[c];
    keys[i] = uint32_t(c);
    vals[i] = int32_t(i);
    atomicAdd(ccount + c, 1);
}

// sorted operand rows and key norms (+inf beyond n)
__global__ void gather_kernel(const __nv_bfloat16 *__restrict__ H, int kh,
                              const float *__restrict__ ny, const int32_t *__restrict__ perm,
                              int64_t n, int64_t npad, __nv_bfloat16 *__restrict__ Hs,
                              float *__restrict__ nys) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= npad) return;
    if (r >= n) {
        if (lane == 0) nys[r] = __int_as_float(0x7f800000);
        return;
    }
    const int64_t i = perm[r];
    if (lane == 0) nys[r] = ny[i];
    const uint4 *src = reinterpret_cast<const uint4 *>(H + i * kh);
    uint4 *dst = reinterpret_cast<uint4 *>(Hs + r * kh);
    for (int q = lane; q < kh / 8; q += 32) dst[q] = src[q];
}

// FP32 rows in sorted order (for the re-rank), float4 when aligned
__global__ void gather_f32_kernel(const float *__restrict__ X, int d,
                                  const int32_t *__restrict__ perm, int64_t n,
                                  float *__restrict__ Xs) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *src = X + int64_t(perm[r]) * d;
    float *dst = Xs + r * d;
    if ((d & 3) == 0 && ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Xs)) & 15) == 0) {
        for (int q = lane; q < d / 4; q += 32)
            reinterpret_cast<float4 *>(dst)[q] = __ldg(reinterpret_cast<const float4 *>(src) + q);
    } else {
        for (int t = lane; t < d; t += 32) dst[t] = __ldg(src + t);
    }
}

// R_c: upper bound on the distance of every member of cell c to its pivot
// (members read from the sorted copy Xs, pivots from X)
template <int FR>
__global__ void radius_kernel(const float *__restrict__ X, const float *__restrict__ Xs, int d,
                              int64_t n, const uint32_t *__restrict__ skey,
                              const int32_t *__restrict__ piv, const int32_t *__restrict__ order,
                              float rho, unsigned *__restrict__ R_bits) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int c = int(skey[r]);
    const float s = warp_sqdist1<FR>(Xs + r * d, X + int64_t(piv[order[c]]) * d, d, lane);
    if (lane == 0) {
        const float h = __fmul_ru(__fsqrt_ru(sq_hi(s, rho)), 1.0f + 0x1p-22f);
        atomicMax(R_bits + c, __float_as_uint(h));
    }
}

// tau_Q: upper bound on the k-th neighbour distance of every row of query
// tile Q, from k other points next to each row in the sorted order, taken
// inside the row's group of cells when the group holds k + 1 points
template <int G>
__global__ void tau_kernel(const float *__restrict__ Xs, int d, int64_t n, int k,
                           const uint32_t *__restrict__ skey,
                           const int32_t *__restrict__ cstart, const int32_t *__restrict__ gfirst,
                           const int32_t *__restrict__ glast, float rho,
                           unsigned *__restrict__ tau_bits, float *__restrict__ tau_row) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int c = int(skey[r]);
    const int64_t cs = cstart[gfirst[c]], ce = cstart[glast[c] + 1];
    int64_t lo, hi;
    if (ce - cs >= k + 1) {
        lo = cs;
        hi = ce - (k + 1);
    } else {
        lo = 0;
        hi = n - (k + 1);
    }
    int64_t w0 = r - k / 2;
    w0 = w0 < lo ? lo : (w0 > hi ? hi : w0);
    // rows of the sorted copy: the row itself and its k + 1 window neighbours
    // sit next to each other in memory
    float4 fx[4];
    row_slices_g<G, 4>(Xs + r * d, d >> 2, lane, fx);
    // the window w0 .. w0 + k always holds r (w0 <= r <= w0 + k), so its
    // other k positions are the candidates: candidate idx sits at w0 + idx,
    // or one further on from r
    float t = 0.0f;
    for (int base = 0; base < k; base += 32) {
        const int idx = base + lane;
        const int64_t pos = w0 + idx + (w0 + idx >= r ? 1 : 0);
        const int cand = idx < k ? int(pos) : -1;
        const float s = warp_sqdist32g<G, 4>(Xs, d, fx, int(r), cand, lane);
        if (cand >= 0) t = fmaxf(t, __fmul_ru(__fsqrt_ru(sq_hi(s, rho)), 1.0f + 0x1p-22f));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) {
        atomicMax(tau_bits + r / QT, __float_as_uint(t));
        tau_row[r] = t;
    }
}

// DP[a][b] <= |p_a - p_b| for b >= a (the upper triangle; dp_mirror_kernel
// copies it to the lower one): warp per (a, 32 consecutive b)
template <int G>
__global__ void pivot_dist_kernel(const float *__restrict__ X, int d, int K,
                                  const int32_t *__restrict__ piv, float rho,
                                  float *__restrict__ DP) {
    const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nbb = (K + 31) / 32;
    if (w >= int64_t(K) * nbb) return;
    const int a = int(w / nbb);
    const int bb = int(w % nbb);
    if (bb * 32 + 31 < a) return;   // the whole block lies below the diagonal
    const int b = bb * 32 + lane;
    const int pa = piv[a];
    float4 fx[4];
    row_slices_g<G, 4>(X + int64_t(pa) * d, d >> 2, lane, fx);
    const int cand = b < K ? piv[b] : -1;
    const float s = warp_sqdist32g<G, 4>(X, d, fx, pa, cand, lane);
    if (b < K && b >= a)
        DP[int64_t(a) * K + b] =
            a == b ? 0.0f : __fmul_rd(__fsqrt_rd(sq_lo(s, rho)), 1.0f - 0x1p-22f);
}

// DP[b][a] = DP[a][b] for b > a: 32 x 32 tiles of the upper triangle,
// transposed through shared memory (coalesced on both sides)
__global__ void dp_mirror_kernel(float *__restrict__ DP, int K) {
    __shared__ float tile[32][33];
    const int ta = blockIdx.y, tb = blockIdx.x;   // tile rows a, columns b
    if (tb < ta) return;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int a = ta * 32 + r, b = tb * 32 + tx;
        tile[r][tx] = (a < K && b < K) ? DP[int64_t(a) * K + b] : 0.0f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int b = tb * 32 + r, a = ta * 32 + tx;   // write row b, column a
        if (a < K && b < K && b > a) DP[int64_t(b) * K + a] = tile[tx][r];
    }
}

// Boruvka step on the complete pivot graph: nearest pivot of another
// component under (DP, id), one warp per pivot
__global__ void pivot_nearest_kernel(const float *__restrict__ DP, int K,
                                     const int32_t *__restrict__ comp, int32_t *__restrict__ nb,
                                     float *__restrict__ nw) {
    const int64_t a = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= K) return;
    const int ca = comp[a];
    uint64_t best = KEY_NONE;
    for (int b = lane; b < K; b += 32) {
        if (comp[b] == ca) continue;
        const uint64_t key = nb_key(DP[a * K + b], uint32_t(b));
        best = key < best ? key : best;
    }
    best = warp_min_u64(best);
    if (lane == 0) {
        nb[a] = best == KEY_NONE ? int32_t(a) : int32_t(key_lo(best));
        nw[a] = best == KEY_NONE ? __int_as_float(0x7f800000) : key_w(best);
    }
}

// DPr[a][b] = DP[order[a]][order[b]] (cells in rank order)
__global__ void dp_gather_kernel(const float *__restrict__ DP, int K,
                                 const int32_t *__restrict__ order, float *__restrict__ DPr) {
    const int64_t a = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= K) return;
    const float *src = DP + int64_t(order[a]) * K;
    for (int b = lane; b < K; b += 32) DPr[a * K + b] = src[order[b]];
}

// Parts of every query tile and key tile: the range of its cells, or, when
// it spans more than NPMAX cells, one ball around the pivot of its middle
// row's cell (cell range = that cell alone; its radius comes from
// tile_radius_kernel, -1 meanwhile; Rt = -2 marks a tile of few cells)
__global__ void tile_cells_kernel(const uint32_t *__restrict__ skey, int64_t n, int64_t nq,
                                  int64_t nk, int32_t *__restrict__ qc, int32_t *__restrict__ kc,
                                  float *__restrict__ qR, float *__restrict__ kR) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < nq) {
        const int64_t r0 = t * QT, r1 = (r0 + QT < n ? r0 + QT : n) - 1;
        int32_t c0 = int32_t(skey[r0]), c1 = int32_t(skey[r1]);
        const bool open = c1 - c0 + 1 > NPMAX;
        if (open) c0 = c1 = int32_t(skey[(r0 + r1) / 2]);
        qc[2 * t] = c0;
        qc[2 * t + 1] = c1;
        qR[t] = open ? 0.0f : -2.0f;
    }
    if (t < nk) {
        const int64_t r0 = t * KT, r1 = (r0 + KT < n ? r0 + KT : n) - 1;
        int32_t c0 = int32_t(skey[r0]), c1 = int32_t(skey[r1]);
        const bool open = c1 - c0 + 1 > NPMAX;
        if (open) c0 = c1 = int32_t(skey[(r0 + r1) / 2]);
        kc[2 * t] = c0;
        kc[2 * t + 1] = c1;
        kR[t] = open ? 0.0f : -2.0f;
    }
}

// Ball radius of every open tile: the largest distance (rounded up) of its
// rows to its centre pivot, one warp per sorted row
template <int FR>
__global__ void tile_radius_kernel(const float *__restrict__ X, const float *__restrict__ Xs,
                                   int d, int64_t n, const int32_t *__restrict__ piv,
                                   const int32_t *__restrict__ order,
                                   const int32_t *__restrict__ qc, const int32_t *__restrict__ kc,
                                   float rho, float *__restrict__ qR, float *__restrict__ kR) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int64_t q = r / QT, t = r / KT;
    const float *x = Xs + r * d;
    if (qR[q] > -1.0f) {
        const float s = warp_sqdist1<FR>(x, X + int64_t(piv[order[qc[2 * q]]]) * d, d, lane);
        if (lane == 0)
            atomicMax(reinterpret_cast<unsigned *>(qR) + q,
                      __float_as_uint(__fmul_ru(__fsqrt_ru(sq_hi(s, rho)), 1.0f + 0x1p-22f)));
    }
    if (kR[t] > -1.0f) {
        const float s = warp_sqdist1<FR>(x, X + int64_t(piv[order[kc[2 * t]]]) * d, d, lane);
        if (lane == 0)
            atomicMax(reinterpret_cast<unsigned *>(kR) + t,
                      __float_as_uint(__fmul_ru(__fsqrt_ru(sq_hi(s, rho)), 1.0f + 0x1p-22f)));
    }
}

// Visit order inside every query tile's list: nearest key tiles first (by
// the smallest pivot distance between their cells, then tile index), so the
// candidate lists of the tile kernel fill with near points early and its
// thresholds reject most keys of the later tiles. The set of tiles is the
// same; lists longer than KLIST_SORT_MAX keep their ascending order.
constexpr int KLIST_SORT_MAX = 4096;   // 32 KB of keys in shared memory
__global__ void __launch_bounds__(256) klist_sort_kernel(const int32_t *__restrict__ off,
                                                         const float *__restrict__ kkey,
                                                         int32_t *__restrict__ klist) {
    __shared__ unsigned long long sk[KLIST_SORT_MAX];
    const int Q = blockIdx.x;
    const int s0 = off[Q], len = off[Q + 1] - s0;
    if (len <= 1 || len > KLIST_SORT_MAX) return;
    int npow = 1;
    while (npow < len) npow <<= 1;
    // keys are distances >= 0: their bit patterns order like the values
    for (int x = threadIdx.x; x < npow; x += blockDim.x)
        sk[x] = x < len ? (uint64_t(__float_as_uint(kkey[s0 + x])) << 32) | uint32_t(klist[s0 + x])
                        : ~0ull;
    __syncthreads();
    for (int size = 2; size <= npow; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int x = threadIdx.x; x < npow; x += blockDim.x) {
                const int y = x ^ stride;
                if (y > x) {
                    const bool asc = (x & size) == 0;
                    const unsigned long long a = sk[x], b = sk[y];
                    if ((a > b) == asc) {
                        sk[x] = b;
                        sk[y] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int x = threadIdx.x; x < len; x += blockDim.x) klist[s0 + x] = int32_t(uint32_t(sk[x]));
}

// Per query tile (one block): which key tiles to visit. FILL = false counts
// them into cnt[Q]; FILL = true writes them (ascending; klist_sort_kernel
// then orders them nearest first) at klist + off[Q], with their sort keys,
// and the smallest lower bound of the skipped tiles into skipQ[Q].
template <bool FILL>
__global__ void __launch_bounds__(256)
tile_pairs_kernel(const int32_t *__restrict__ qc, const int32_t *__restrict__ kc,
                  const float *__restrict__ qR, const float *__restrict__ kR, int64_t nk,
                  int K, const float *__restrict__ DP, const float *__restrict__ R,
                  const float *__restrict__ tauQ, float margin, int32_t *__restrict__ cnt,
                  const int32_t *__restrict__ off, int32_t *__restrict__ klist,
                  float *__restrict__ kkey, float *__restrict__ skipQ) {
    __shared__ int wsum[8];
    __shared__ float wmin[8];
    __shared__ int base_s;
    const int Q = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a0 = qc[2 * Q], a1 = qc[2 * Q + 1];
    const float qball = qR[Q];   // >= 0: one ball for the whole tile
    const float tau = __fmul_ru(tauQ[Q], margin);
    const float inf = __int_as_float(0x7f800000);
    float ra[NPMAX];
#pragma unroll
    for (int q = 0; q < NPMAX; ++q) ra[q] = a0 + q <= a1 ? (qball >= 0.0f ? qball : R[a0 + q]) : 0.0f;
    int count = 0;
    float smin = inf;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nk; c0 += 256) {
        const int64_t T = c0 + threadIdx.x;
        bool visit = false;
        float lb = inf, dmin = inf;
        if (T < nk) {
            const int b0 = kc[2 * T], b1 = kc[2 * T + 1];
            const float kball = kR[T];
#pragma unroll
            for (int q = 0; q < NPMAX; ++q) {
                if (a0 + q > a1) break;
                const float *dp = DP + int64_t(a0 + q) * K;
                for (int b = b0; b <= b1; ++b) {
                    lb = fminf(lb, __fsub_rd(__fsub_rd(dp[b], ra[q]), kball >= 0.0f ? kball : R[b]));
                    dmin = fminf(dmin, dp[b]);
                }
            }
            visit = !(lb > tau);
            if (!visit) smin = fminf(smin, lb);
        }
        if constexpr (FILL) {
            const unsigned bal = __ballot_sync(0xffffffffu, visit);
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            int pre = base_s;
            for (int w = 0; w < warp; ++w) pre += wsum[w];
            if (visit) {
                const int at = off[Q] + pre + __popc(bal & ((1u << lane) - 1u));
                klist[at] = int32_t(T);
                kkey[at] = dmin;   // nearest pivot pair of the two tiles' cells
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int s = 0;
                for (int w = 0; w < 8; ++w) s += wsum[w];
                base_s += s;
            }
            __syncthreads();
        } else {
            count += visit ? 1 : 0;
        }
    }
    if constexpr (FILL) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) smin = fminf(smin, __shfl_xor_sync(0xffffffffu, smin, o));
        if (lane == 0) wmin[warp] = smin;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = inf;
            for (int w = 0; w < 8; ++w) m = fminf(m, wmin[w]);
            skipQ[Q] = m;
        }
    } else {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
        if (lane == 0) wsum[warp] = count;
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += wsum[w];
            cnt[Q] = s;
        }
    }
}

// Exclusive scan of three counters over the block (blockDim.x a multiple of
// 32): every thread's v becomes the sum of the lower threads' values.
__device__ __forceinline__ void block_scan3(int3 &v) {
    __shared__ int3 wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int3 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, inc.x, o);
        const int b = __shfl_up_sync(0xffffffffu, inc.y, o);
        const int c = __shfl_up_sync(0xffffffffu, inc.z, o);
        if (lane >= o) {
            inc.x += a;
            inc.y += b;
            inc.z += c;
        }
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int3 w = lane < nw ? wsum[lane] : make_int3(0, 0, 0);
        int3 wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, wi.x, o);
            const int b = __shfl_up_sync(0xffffffffu, wi.y, o);
            const int c = __shfl_up_sync(0xffffffffu, wi.z, o);
            if (lane >= o) {
                wi.x += a;
                wi.y += b;
                wi.z += c;
            }
        }
        if (lane < nw) wsum[lane] = make_int3(wi.x - w.x, wi.y - w.y, wi.z - w.z);
    }
    __syncthreads();
    const int3 wb = wsum[warp];
    v = make_int3(wb.x + inc.x - v.x, wb.y + inc.y - v.y, wb.z + inc.z - v.z);
    __syncthreads();
}

// Work items of the pruned tile kernel (one block of 1024 threads). A query
// tile whose key list is longer than L = max(PRUNE_SPLIT_MIN, ceil(visited /
// PRUNE_SPLIT_TILES)) becomes ceil(len / L) parts of near-equal length, each
// its own item with a side slot for its rows' candidates; the parts come
// first (the longest work starts first), then the whole lists in tile
// order. The counts are bounded: fewer than PRUNE_SPLIT_TILES lists are
// longer than L, and their parts number fewer than visited / L plus that
// count, i.e. fewer than PRUNE_SPLIT_SLOTS. Were the bound to fail, nothing
// would be split.
__global__ void __launch_bounds__(1024)
split_table_kernel(const int32_t *__restrict__ off, int64_t nq, int nkb, int64_t n,
                   const int32_t *__restrict__ visited, TcTile *__restrict__ tab,
                   int32_t *__restrict__ nitems, int32_t *__restrict__ splitq,
                   int32_t *__restrict__ nsplit) {
    __shared__ int3 totals;
    const int64_t per = (nq + blockDim.x - 1) / blockDim.x;
    const int64_t q0 = min(nq, int64_t(threadIdx.x) * per), q1 = min(nq, q0 + per);
    const int64_t vis = *visited;
    int64_t L = (vis + PRUNE_SPLIT_TILES - 1) / PRUNE_SPLIT_TILES;
    if (L < PRUNE_SPLIT_MIN) L = PRUNE_SPLIT_MIN;
    for (int attempt = 0; attempt < 2; ++attempt) {
        int3 c = make_int3(0, 0, 0);   // parts, whole lists, split lists
        for (int64_t q = q0; q < q1; ++q) {
            const int64_t len = off[q + 1] - off[q];
            if (len > L) {
                c.x += int((len + L - 1) / L);
                c.z += 1;
            } else {
                c.y += 1;
            }
        }
        int3 pre = c;
        block_scan3(pre);
        if (threadIdx.x == blockDim.x - 1) totals = make_int3(pre.x + c.x, pre.y + c.y, pre.z + c.z);
        __syncthreads();
        const int3 tot = totals;
        __syncthreads();
        if (tot.x > PRUNE_SPLIT_SLOTS || tot.z > PRUNE_SPLIT_TILES) {
            L = int64_t(1) << 40;   // split nothing (uniform: every thread saw the same totals)
            continue;
        }
        int pi = pre.x, wi = tot.x + pre.y, si = pre.z;
        for (int64_t q = q0; q < q1; ++q) {
            const int kt0 = off[q], kt1 = off[q + 1];
            const int64_t len = kt1 - kt0;
            TcTile t;
            t.q0 = int(q * QT);
            t.nkb = nkb;
            t.row_end = int(n);
            t.shift = 0;
            if (len > L) {
                const int P = int((len + L - 1) / L);
                splitq[3 * si] = int(q);
                splitq[3 * si + 1] = pi;
                splitq[3 * si + 2] = P;
                ++si;
                for (int p = 0; p < P; ++p) {
                    t.kt0 = kt0 + int(len * p / P);
                    t.kt1 = kt0 + int(len * (p + 1) / P);
                    t.part = pi + 1;
                    tab[pi++] = t;
                }
            } else {
                t.kt0 = kt0;
                t.kt1 = kt1;
                t.part = 0;
                tab[wi++] = t;
            }
        }
        if (threadIdx.x == 0) {
            *nitems = tot.x + tot.y;
            *nsplit = tot.z;
        }
        return;
    }
}

// Order of the cells. The minimum spanning tree of the pivots is cut at
// edges longer than twice its median edge into groups (single linkage);
// groups are laid out one after another, each by a depth-first walk over
// its short edges, shortest first. Cells next to each other in the order
// are then close, and every group is one contiguous run. Output (4 K ints):
// order[rank] = pivot, rank[pivot], and per rank the first and last rank of
// its group.
void order_cells(int K, const std::vector<int32_t> &tu, const std::vector<int32_t> &tv,
                 const std::vector<float> &tw, int32_t *out) {
    const size_t m = tu.size();
    std::vector<float> ws(tw);
    float theta = 0.0f;
    if (m > 0) {
        std::nth_element(ws.begin(), ws.begin() + m / 2, ws.end());
        theta = 2.0f * ws[m / 2];
    }
    std::vector<std::vector<std::pair<float, int32_t>>> adj(static_cast<size_t>(K));
    for (size_t e = 0; e < m; ++e) {
        adj[size_t(tu[e])].push_back({tw[e], tv[e]});
        adj[size_t(tv[e])].push_back({tw[e], tu[e]});
    }
    for (auto &l : adj) std::sort(l.begin(), l.end());
    int32_t *order = out, *rank = out + K, *gfirst = out + 2 * K, *glast = out + 3 * K;
    std::vector<char> seen(static_cast<size_t>(K), 0);
    std::vector<int32_t> groups, stack;
    int32_t pos = 0;
    for (int32_t root = 0; root < K; ++root) {   // every tree component (the forest case too)
        if (seen[size_t(root)]) continue;
        seen[size_t(root)] = 1;
        groups.push_back(root);
        while (!groups.empty()) {
            const int32_t g = groups.back();
            groups.pop_back();
            const int32_t first = pos;
            stack.push_back(g);
            while (!stack.empty()) {
                const int32_t u = stack.back();
                stack.pop_back();
                order[pos++] = u;
                const auto &l = adj[size_t(u)];
                for (size_t q = l.size(); q-- > 0;) {   // shortest edge popped first
                    const int32_t v = l[q].second;
                    if (seen[size_t(v)]) continue;
                    seen[size_t(v)] = 1;
                    if (l[q].first <= theta) stack.push_back(v);
                    else groups.push_back(v);
                }
            }
            for (int32_t r = first; r < pos; ++r) {
                gfirst[r] = first;
                glast[r] = pos - 1;
            }
        }
    }
    for (int32_t r = 0; r < K; ++r) rank[order[r]] = r;
}

}  // namespace

int prune_pivots(int64_t n) {
    int64_t K = n / 256;
    if (K < 16) K = 16;
    if (K > 4096) K = 4096;
    return int(K);
}

int prune_extra(int64_t n) { return prune_pivots(n) / 2; }

int prune_pivots_max(int64_t n) { return prune_pivots(n) + 2 * prune_extra(n); }

bool prune_supported(int64_t n, int d, int k, bool vec4) {
    // the per-query-tile list offsets are int32: every (query tile, key tile)
    // pair must be countable, whatever fraction is visited
    const int64_t nq = (n + QT - 1) / QT, nk = (n + KT - 1) / KT;
    return vec4 && d >= 4 && d <= 512 && n >= 4 * int64_t(k + 1) && n >= 4096 &&
           nq * nk < (int64_t(1) << 31);
}

size_t prune_workspace(int64_t n, int d, int kh, int kp, int64_t nq, int64_t nk) {
    const int64_t K = prune_pivots_max(n);
    const int64_t Kpad = (K + KT - 1) / KT * KT;
    size_t b = 0;
    b += align256(size_t(K) * 4) + align256(size_t(K) * kh * 2) + align256(size_t(Kpad) * 4);
    b += align256(size_t(n) * 4) * 2 + align256(size_t(K + 1) * 4) * 2;        // keys, perm, cells
    b += align256(size_t(n) * 4) * 2 + align256(size_t(K) * 4) + radix_sort_workspace(n);  // coverage
    b += radix_sort_workspace(n) + scan_workspace(K + 1) + 256;
    b += align256(size_t(n) * kh * 2) + align256(size_t(nk) * KT * 4);         // sorted operand
    b += align256(size_t(K) * 4) + align256(size_t(nq) * 4);                   // R, tau
    b += align256(size_t(n) * 4);                                              // tau per row
    b += align256(size_t(K) * K * 4) * 2;                                      // DP, DPr
    b += align256(size_t(4 * K) * 4) + align256(size_t(K) * 4) * 5;             // order, tree
    b += boruvka_workspace(K);                                                 // pivot tree
    b += align256(size_t(nq) * 8) + align256(size_t(nk) * 8);                  // tile cells
    b += align256(size_t(nq) * 4) + align256(size_t(nk) * 4);                  // tile balls
    b += align256(size_t(nq + 1) * 4) * 2 + scan_workspace(nq + 1) + 256;      // counts, offsets
    b += align256(size_t(nq) * nk * 4) * 2;                                    // lists, keys (worst case)
    b += align256(size_t(nq) * 4) +
         align256(size_t(nq + PRUNE_SPLIT_SLOTS) * sizeof(TcTile));           // skip, work items
    b += align256(4) * 2 + align256(size_t(3) * PRUNE_SPLIT_TILES * 4);        // item and split counts
    b += align256(size_t(PRUNE_SPLIT_SLOTS) * QT * kp * 4) * 2 +
         align256(size_t(PRUNE_SPLIT_SLOTS) * QT * 4);                         // parts' candidates
    b += align256(size_t(n) * kp * 4) + align256(size_t(n) * 4);               // sorted outputs
    b += align256(size_t(n) * d * 4);                                          // sorted points
    return b;
}

famst_status prune_pivot_operands(const Exec &ex, const __nv_bfloat16 *H, int kh, const float *ny,
                                  int64_t n, int K, int Kpad, int32_t *piv, __nv_bfloat16 *Hp,
                                  float *nyp) {
    FAMST_LAUNCH(ex, pivots_kernel, nblk(int64_t(Kpad) * 32, 256), 256, 0, H, kh, ny, n, K, Kpad,
                 nullptr, piv, Hp, nyp);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

// Coverage: M points spread over those far from their current pivot
// (approximate distances of the top-1 pass) become pivots K .. K + M - 1. A
// group of points with no pivot of its own sits far from every pivot, so it
// gains some; without them its points would widen foreign cells' balls.
famst_status prune_augment(const Exec &ex, Arena &ar, const float *xn2, const float *s1, int64_t n,
                           const __nv_bfloat16 *H, int kh, const float *ny, int M, int K,
                           int32_t *piv, __nv_bfloat16 *Hp, float *nyp, int *me) {
    const size_t mark = ar.off;
    uint32_t *keys = ar.take<uint32_t>(size_t(n));
    int32_t *vals = ar.take<int32_t>(size_t(n));
    int32_t *rows = ar.take<int32_t>(size_t(M));
    int32_t *me_dev = ar.take<int32_t>(1);
    if (!keys || !vals || !rows || !me_dev) return FAMST_ERR_OOM;
    FAMST_LAUNCH(ex, far_key_kernel, nblk(n, 256), 256, 0, xn2, s1, n, keys, vals);
    famst_status st = radix_sort_pairs(ex, ar, keys, vals, n, 32);
    if (st == FAMST_OK) {
        FAMST_LAUNCH(ex, far_pick_kernel, 1, 256, 0, keys, vals, n, M, rows, me_dev);
        FAMST_LAUNCH(ex, pivots_kernel, nblk(int64_t(M) * 32, 256), 256, 0, H, kh, ny, n, M, M,
                     rows, piv + K, Hp + size_t(K) * kh, nyp + K);
        // the number of distinct new pivots (the other slots repeat one point)
        int32_t h = 0;
        if (cudaMemcpyAsync(&h, me_dev, 4, cudaMemcpyDeviceToHost, ex.stream) != cudaSuccess ||
            cudaStreamSynchronize(ex.stream) != cudaSuccess)
            st = FAMST_ERR_CUDA;
        *me = h;
    }
    ar.off = mark;
    if (st != FAMST_OK) return st;
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

famst_status prune_partition(const Exec &ex, Arena &ar, const float *X, int d, int64_t n, int k,
                             const __nv_bfloat16 *H, int kh, const float *ny, int nkb, int K,
                             const int32_t *piv, const int32_t *acand, int akp,
                             int32_t *pinned_host, PruneOut *out) {
    const int64_t nq = (n + QT - 1) / QT, nk = (n + KT - 1) / KT;
    uint32_t *keys = ar.take<uint32_t>(size_t(n));
    int32_t *perm = ar.take<int32_t>(size_t(n));
    int32_t *ccount = ar.take<int32_t>(size_t(K + 1));
    int32_t *cstart = ar.take<int32_t>(size_t(K + 1));
    __nv_bfloat16 *Hs = ar.take<__nv_bfloat16>(size_t(n) * kh);
    float *nys = ar.take<float>(size_t(nk) * KT);
    float *R = ar.take<float>(size_t(K));
    float *tauQ = ar.take<float>(size_t(nq));
    float *tau_row = ar.take<float>(size_t(n));
    float *DP = ar.take<float>(size_t(K) * K);
    float *DPr = ar.take<float>(size_t(K) * K);
    int32_t *ord = ar.take<int32_t>(size_t(4) * K);   // order, rank, gfirst, glast
    int32_t *tu = ar.take<int32_t>(size_t(K));
    int32_t *tv = ar.take<int32_t>(size_t(K));
    float *tw = ar.take<float>(size_t(K));
    int32_t *nb = ar.take<int32_t>(size_t(K));
    float *nw = ar.take<float>(size_t(K));
    int32_t *qc = ar.take<int32_t>(size_t(nq) * 2);
    int32_t *kc = ar.take<int32_t>(size_t(nk) * 2);
    float *qR = ar.take<float>(size_t(nq));
    float *kR = ar.take<float>(size_t(nk));
    int32_t *cnt = ar.take<int32_t>(size_t(nq + 1));
    int32_t *off = ar.take<int32_t>(size_t(nq + 1));
    int32_t *klist = ar.take<int32_t>(size_t(nq) * nk);
    float *kkey = ar.take<float>(size_t(nq) * nk);
    float *skipQ = ar.take<float>(size_t(nq));
    TcTile *tab = ar.take<TcTile>(size_t(nq + PRUNE_SPLIT_SLOTS));
    int32_t *nitems = ar.take<int32_t>(1);
    int32_t *nsplit = ar.take<int32_t>(1);
    int32_t *splitq = ar.take<int32_t>(size_t(3) * PRUNE_SPLIT_TILES);
    int32_t *total = ar.take<int32_t>(1);
    float *Xs = ar.take<float>(size_t(n) * d);
    if (!Xs) return FAMST_ERR_OOM;
    if (!keys || !perm || !ccount || !cstart || !Hs || !nys || !R || !tauQ || !tau_row || !DP ||
        !DPr || !ord ||
        !tu || !tv || !tw || !nb || !nw || !qc || !kc || !qR || !kR || !cnt || !off || !klist ||
        !kkey || !skipQ || !tab || !nitems || !nsplit || !splitq ||
        !total)
        return FAMST_ERR_OOM;
    const float rho = fast_rho(d, 4);
    if (cudaMemsetAsync(ccount, 0, size_t(K + 1) * 4, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, size_t(nq + 1) * 4, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(R, 0, size_t(K) * 4, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(tauQ, 0, size_t(nq) * 4, ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    const int64_t nbb = (K + 31) / 32;
    const int fr = d <= 128 ? 1 : (d <= 256 ? 2 : 4);
    const int G = sq_group(d);
    // 1. pivot distances (lower bounds; computed once per unordered pair)
    const unsigned pgrid = nblk(int64_t(K) * nbb * 32, 256);
    switch (G) {
        case 2: FAMST_LAUNCH(ex, pivot_dist_kernel<2>, pgrid, 256, 0, X, d, K, piv, rho, DP); break;
        case 4: FAMST_LAUNCH(ex, pivot_dist_kernel<4>, pgrid, 256, 0, X, d, K, piv, rho, DP); break;
        case 8: FAMST_LAUNCH(ex, pivot_dist_kernel<8>, pgrid, 256, 0, X, d, K, piv, rho, DP); break;
        case 16: FAMST_LAUNCH(ex, pivot_dist_kernel<16>, pgrid, 256, 0, X, d, K, piv, rho, DP); break;
        default: FAMST_LAUNCH(ex, pivot_dist_kernel<32>, pgrid, 256, 0, X, d, K, piv, rho, DP);
    }
    {
        const unsigned nt = unsigned((K + 31) / 32);
        FAMST_LAUNCH(ex, dp_mirror_kernel, dim3(nt, nt), dim3(32, 8), 0, DP, K);
    }
    // 2. order of the cells: minimum spanning tree of the pivots (Boruvka)
    famst_status st;
    {
        const size_t mark = ar.off;
        BvState S;
        st = bv_state_init(ex, ar, K, &S);
        S.knn_exact = true;   // nb / nw: each pivot's exact nearest under (DP, id)
        int64_t got = 0;
        for (int r = 0; r < 64 && got < K - 1 && st == FAMST_OK; ++r) {
            FAMST_LAUNCH(ex, pivot_nearest_kernel, nblk(int64_t(K) * 32, 256), 256, 0, DP, K,
                         S.comp, nb, nw);
            st = bv_round(ex, ar, S, nb, nw, 1, nullptr, nullptr, nullptr, 0, MstOut{tu, tv, tw},
                          got, pinned_host);
            if (st != FAMST_OK) break;
            if (*pinned_host == 0) break;
            got += *pinned_host;
        }
        ar.off = mark;
        if (st != FAMST_OK) return st;
        std::vector<int32_t> hu(static_cast<size_t>(got)), hv(static_cast<size_t>(got));
        std::vector<float> hw(static_cast<size_t>(got));
        if (got > 0 &&
            (cudaMemcpyAsync(hu.data(), tu, size_t(got) * 4, cudaMemcpyDeviceToHost, ex.stream) !=
                 cudaSuccess ||
             cudaMemcpyAsync(hv.data(), tv, size_t(got) * 4, cudaMemcpyDeviceToHost, ex.stream) !=
                 cudaSuccess ||
             cudaMemcpyAsync(hw.data(), tw, size_t(got) * 4, cudaMemcpyDeviceToHost, ex.stream) !=
                 cudaSuccess ||
             cudaStreamSynchronize(ex.stream) != cudaSuccess))
            return FAMST_ERR_CUDA;
        std::vector<int32_t> h_ord(static_cast<size_t>(4) * K);
        order_cells(K, hu, hv, hw, h_ord.data());
        if (cudaMemcpyAsync(ord, h_ord.data(), size_t(4) * K * 4, cudaMemcpyHostToDevice,
                            ex.stream) != cudaSuccess ||
            cudaStreamSynchronize(ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
    }
    const int32_t *order = ord, *rank = ord + K, *gfirst = ord + 2 * K, *glast = ord + 3 * K;
    // 3. cells in rank order, sorted points
    FAMST_LAUNCH(ex, assign_kernel, nblk(n, 256), 256, 0, acand, akp, n, K, rank, keys, perm,
                 ccount);
    int bits = 0;
    while ((int64_t(1) << bits) < K) ++bits;
    {
        const size_t mark = ar.off;
        st = radix_sort_pairs(ex, ar, keys, perm, n, bits);
        if (st == FAMST_OK) st = exclusive_scan_i32(ex, ar, ccount, cstart, K + 1, total);
        ar.off = mark;
        if (st != FAMST_OK) return st;
    }
    FAMST_LAUNCH(ex, gather_kernel, nblk(nk * KT * 32, 256), 256, 0, H, kh, ny, perm, n, nk * KT,
                 Hs, nys);
    FAMST_LAUNCH(ex, gather_f32_kernel, nblk(n * 32, 256), 256, 0, X, d, perm, n, Xs);
    FAMST_LAUNCH(ex, dp_gather_kernel, nblk(int64_t(K) * 32, 256), 256, 0, DP, K, order, DPr);
    // 4. balls and radii of interest
    const unsigned wgrid = nblk(n * 32, 256);
    if (fr == 1)
        FAMST_LAUNCH(ex, radius_kernel<1>, wgrid, 256, 0, X, Xs, d, n, keys, piv, order, rho,
                     reinterpret_cast<unsigned *>(R));
    else if (fr == 2)
        FAMST_LAUNCH(ex, radius_kernel<2>, wgrid, 256, 0, X, Xs, d, n, keys, piv, order, rho,
                     reinterpret_cast<unsigned *>(R));
    else
        FAMST_LAUNCH(ex, radius_kernel<4>, wgrid, 256, 0, X, Xs, d, n, keys, piv, order, rho,
                     reinterpret_cast<unsigned *>(R));
#define TAU(GG)                                                                                  \
    FAMST_LAUNCH(ex, tau_kernel<GG>, wgrid, 256, 0, Xs, d, n, k, keys, cstart, gfirst, glast,     \
                 rho, reinterpret_cast<unsigned *>(tauQ), tau_row)
    switch (G) {
        case 2: TAU(2); break;
        case 4: TAU(4); break;
        case 8: TAU(8); break;
        case 16: TAU(16); break;
        default: TAU(32);
    }
#undef TAU
    // 5. lists
    FAMST_LAUNCH(ex, tile_cells_kernel, nblk(nq > nk ? nq : nk, 256), 256, 0, keys, n, nq, nk, qc,
                 kc, qR, kR);
    if (fr == 1)
        FAMST_LAUNCH(ex, tile_radius_kernel<1>, wgrid, 256, 0, X, Xs, d, n, piv, order, qc, kc,
                     rho, qR, kR);
    else if (fr == 2)
        FAMST_LAUNCH(ex, tile_radius_kernel<2>, wgrid, 256, 0, X, Xs, d, n, piv, order, qc, kc,
                     rho, qR, kR);
    else
        FAMST_LAUNCH(ex, tile_radius_kernel<4>, wgrid, 256, 0, X, Xs, d, n, piv, order, qc, kc,
                     rho, qR, kR);
    // visit unless LB > tau (1 + margin): the margin covers the canonical
    // rounding on both sides of the certificate's comparison
    const float margin = float(1.0 + 4.0 * (d + 4) * std::ldexp(1.0, -24) + std::ldexp(1.0, -20));
    FAMST_LAUNCH(ex, tile_pairs_kernel<false>, unsigned(nq), 256, 0, qc, kc, qR, kR, nk, K, DPr, R,
                 tauQ, margin, cnt, nullptr, nullptr, nullptr, nullptr);
    {
        const size_t mark = ar.off;
        st = exclusive_scan_i32(ex, ar, cnt, off, nq + 1, total);
        ar.off = mark;
        if (st != FAMST_OK) return st;
    }
    FAMST_LAUNCH(ex, tile_pairs_kernel<true>, unsigned(nq), 256, 0, qc, kc, qR, kR, nk, K, DPr, R,
                 tauQ, margin, nullptr, off, klist, kkey, skipQ);
    FAMST_LAUNCH(ex, klist_sort_kernel, unsigned(nq), 256, 0, off, kkey, klist);
    FAMST_LAUNCH(ex, split_table_kernel, 1, 1024, 0, off, nq, nkb, n, total, tab, nitems, splitq,
                 nsplit);
    out->perm = perm;
    out->Hs = Hs;
    out->nys = nys;
    out->klist = klist;
    out->tab = tab;
    out->nitems = nitems;
    out->splitq = splitq;
    out->nsplit = nsplit;
    out->skipQ = skipQ;
    out->Xs = Xs;
    out->tau_row = tau_row;
    out->visited = total;
    out->nq = nq;
    out->nk = nk;
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}


}  // namespace famst
