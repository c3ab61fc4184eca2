// Internal declarations shared by the FAMST CUDA translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "famst.h"

namespace famst {

// ------------------------------------------------------------------ host

// Execution environment of one library call: the stream its work goes to
// and the context's launch counter.
// CUDA-event timers around single kernels of a build (the distance tiles,
// the re-rank, Algorithm 3's and Algorithm 4's kernels), read back into the
// build info after the call synchronises.
enum : int { TIMER_TILES = 0, TIMER_RERANK = 1, TIMER_CONNECT = 2, TIMER_REFINE = 3, TIMER_N = 4 };
struct KernelTimers {
    cudaEvent_t ev[2 * TIMER_N] = {};
    bool used[TIMER_N] = {};
};

struct Exec {
    cudaStream_t stream;
    unsigned long long *launches;
    int num_sms;
    int *dstatus;  // device status word (see STATUS_* below)
    int loop_limit = 0;  // iteration limit of the bounded loops; 0 = their defaults
    KernelTimers *timers = nullptr;  // optional
};

// Record the start / end event of timer `slot` on the call's stream.
static inline void timer_mark(const Exec &ex, int slot, bool end) {
    if (!ex.timers) return;
    cudaEventRecord(ex.timers->ev[2 * slot + (end ? 1 : 0)], ex.stream);
    if (end) ex.timers->used[slot] = true;
}

// Bits of the device status word. Kernels OR them in; the host reads the
// word at the next synchronisation point.
enum : int {
    STATUS_NONFINITE = 1,       // a NaN or an infinity in X
    STATUS_REFINE_CAP = 2,      // an edge still changed in sweep max_iters
    STATUS_LOOP_LIMIT = 4,      // a bounded device loop reached its limit
    STATUS_DISCONNECTED = 8,    // Boruvka found no outgoing edge with >1 component left
    STATUS_BAD_ID = 16,         // a vertex id out of range or inconsistent
    STATUS_INTERNAL = 64,       // an internal buffer bound was exceeded (a bug)
};

#define FAMST_LAUNCH(ex, kern, grid, block, smem, ...)                         \
    do {                                                                       \
        kern<<<(grid), (block), (smem), (ex).stream>>>(__VA_ARGS__);           \
        ++*(ex).launches;                                                      \
    } while (0)

// Bump allocator over the context workspace.
struct Arena {
    char *base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        T *p = reinterpret_cast<T *>(base + off);
        off += bytes;
        return p;
    }
};

static inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Shared-memory opt-in of a kernel. Skipped while the stream is being
// captured into a CUDA graph: the attribute persists from the eager run that
// always precedes a capture, and setting it is not a stream operation.
static inline bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive;
}
template <class K>
static inline cudaError_t set_smem_attr(K *kernel, size_t bytes, cudaStream_t s) {
    if (stream_capturing(s)) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

// ---------------------------------------------------------------- device

static constexpr uint64_t KEY_NONE = ~0ull;

// Canonical FP32 distance. 32 partial sums, partial l taking the
// coordinates t = l, l+32, ... < d in increasing order (p_l = fmaf(delta_t,
// delta_t, p_l), delta_t = x_t - y_t), combined by the butterfly o = 16, 8,
// 4, 2, 1 (p_l <- p_l + p_(l xor o)), then a correctly rounded square root.
// A warp evaluates it with lane l holding p_l (canon_p_warp); one thread
// evaluates the identical value with the 32 partials in registers: the
// butterfly's value at lane 0 is the binary tree q_l = p_l + p_(l+16),
// r_l = q_l + q_(l+8), ... over l < 16, 8, 4, 2, 1 (addition commutes).
// VEC = 4 reads float4 (rows 16-byte aligned, d % 4 == 0).
template <int VEC>
__device__ __forceinline__ float canon_p(const float *__restrict__ a,
                                         const float *__restrict__ b, int d) {
    float p[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) p[l] = 0.0f;
    if constexpr (VEC == 4) {
        const float4 *a4 = reinterpret_cast<const float4 *>(a);
        const float4 *b4 = reinterpret_cast<const float4 *>(b);
        const int d4 = d >> 2;
        for (int q0 = 0; q0 < d4; q0 += 8) {   // 32 coordinates: one term per partial
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (q0 + i < d4) {
                    const float4 x = __ldg(a4 + q0 + i), y = __ldg(b4 + q0 + i);
                    const float t0 = __fsub_rn(x.x, y.x), t1 = __fsub_rn(x.y, y.y);
                    const float t2 = __fsub_rn(x.z, y.z), t3 = __fsub_rn(x.w, y.w);
                    p[4 * i + 0] = __fmaf_rn(t0, t0, p[4 * i + 0]);
                    p[4 * i + 1] = __fmaf_rn(t1, t1, p[4 * i + 1]);
                    p[4 * i + 2] = __fmaf_rn(t2, t2, p[4 * i + 2]);
                    p[4 * i + 3] = __fmaf_rn(t3, t3, p[4 * i + 3]);
                }
            }
        }
    } else {
        for (int t0 = 0; t0 < d; t0 += 32) {
#pragma unroll
            for (int l = 0; l < 32; ++l) {
                if (t0 + l < d) {
                    const float t = __fsub_rn(__ldg(a + t0 + l), __ldg(b + t0 + l));
                    p[l] = __fmaf_rn(t, t, p[l]);
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
        for (int l = 0; l < o; ++l) p[l] = __fadd_rn(p[l], p[l + o]);
    }
    return p[0];
}

// The same value computed by a whole warp (every lane gets it): lane l
// accumulates partial l over coalesced loads, then the xor butterfly.
__device__ __forceinline__ float canon_p_warp(const float *__restrict__ a,
                                              const float *__restrict__ b, int d, int lane) {
    float p = 0.0f;
    for (int t = lane; t < d; t += 32) {
        const float x = __fsub_rn(__ldg(a + t), __ldg(b + t));
        p = __fmaf_rn(x, x, p);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
    return p;
}

template <int VEC>
__device__ __forceinline__ float canon_dist(const float *__restrict__ a,
                                            const float *__restrict__ b, int d) {
    return __fsqrt_rn(canon_p<VEC>(a, b, d));
}

// Key of a neighbour candidate: (w, id) lexicographic as one uint64.
// w >= 0, so its IEEE bits order like the value.
__device__ __forceinline__ uint64_t nb_key(float w, uint32_t id) {
    return (uint64_t(__float_as_uint(w)) << 32) | id;
}
__device__ __forceinline__ float key_w(uint64_t k) { return __uint_as_float(uint32_t(k >> 32)); }
__device__ __forceinline__ uint32_t key_lo(uint64_t k) { return uint32_t(k); }

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m) {
    uint32_t lo = uint32_t(v), hi = uint32_t(v >> 32);
    lo = __shfl_xor_sync(0xffffffffu, lo, m);
    hi = __shfl_xor_sync(0xffffffffu, hi, m);
    return (uint64_t(hi) << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl_idx_u64(uint64_t v, int src) {
    uint32_t lo = uint32_t(v), hi = uint32_t(v >> 32);
    lo = __shfl_sync(0xffffffffu, lo, src);
    hi = __shfl_sync(0xffffffffu, hi, src);
    return (uint64_t(hi) << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int delta) {
    uint32_t lo = uint32_t(v), hi = uint32_t(v >> 32);
    lo = __shfl_up_sync(0xffffffffu, lo, delta);
    hi = __shfl_up_sync(0xffffffffu, hi, delta);
    return (uint64_t(hi) << 32) | lo;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        uint64_t o = shfl_xor_u64(v, m);
        v = o < v ? o : v;
    }
    return v;
}

// ---------------------------------------------- fast squared distances
// Warp-cooperative squared distances for filters and bounds (never for a
// stored weight). Rows are 16-byte aligned with d % 4 == 0; lane l holds
// float4 columns l, l + 32, ..., FR of them (d <= 128 FR). Each term is
// fl(y_t - x_t)^2 accumulated by fmaf as in the canonical distance, only in
// another order, so the result is within gamma_n of the exact sum of the
// rounded differences, n = d + 4 FR + 5 roundings at most (the canonical
// chain: gamma_d). fast_rho(d, FR) bounds both ratios p_canon / p_fast and
// S / p_fast (S the exact sum) to [1 - rho, 1 + rho].
inline float fast_rho(int d, int fr) {
    const double u = 1.0 / 16777216.0;
    const double nu = double(d + 4 * fr + 5) * u;
    return float(2.01 * nu / (1.0 - nu) + 4.0 * u);
}

template <int FR>
__device__ __forceinline__ void row_slices(const float *__restrict__ row, int d4, int lane,
                                           float4 (&f)[FR]) {
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const int q = lane + 32 * r;
        f[r] = q < d4 ? __ldg(reinterpret_cast<const float4 *>(row) + q)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int FR>
__device__ __forceinline__ float slice_sq(const float *__restrict__ row, int d4, int lane,
                                          const float4 (&fx)[FR]) {
    float a = 0.0f;
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const int q = lane + 32 * r;
        if (q < d4) {
            const float4 y = __ldg(reinterpret_cast<const float4 *>(row) + q);
            const float t0 = __fsub_rn(y.x, fx[r].x);
            a = __fmaf_rn(t0, t0, a);
            const float t1 = __fsub_rn(y.y, fx[r].y);
            a = __fmaf_rn(t1, t1, a);
            const float t2 = __fsub_rn(y.z, fx[r].z);
            a = __fmaf_rn(t2, t2, a);
            const float t3 = __fsub_rn(y.w, fx[r].w);
            a = __fmaf_rn(t3, t3, a);
        }
    }
    return a;
}

// One pair per warp: squared distance of rows a and b, in every lane.
template <int FR>
__device__ __forceinline__ float warp_sqdist1(const float *__restrict__ a,
                                              const float *__restrict__ b, int d, int lane) {
    float4 fa[FR];
    row_slices<FR>(a, d >> 2, lane, fa);
    float s = slice_sq<FR>(b, d >> 2, lane, fa);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
    return s;
}

// Packed FP32 pairs (sm_100 f32x2 instructions): two lanes of IEEE
// round-to-nearest arithmetic per instruction.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_sqacc(unsigned long long t, unsigned long long a) {
    unsigned long long r;   // t * t + a, each lane one rounding
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(t), "l"(a));
    return r;
}
__device__ __forceinline__ float f2_hsum(unsigned long long a) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
    return __fadd_rn(lo, hi);
}

// Grouped warp-wide fast squared distances. Every candidate row is read by
// a group of G lanes (float4 columns g, g + G, ..., V of them per lane,
// G V 4 >= d), so 32 / G rows are read per load instruction, each
// contiguously. Each lane keeps G partial sums (one per step, in packed FP32
// pairs), a butterfly transpose-sum inside the group gathers each row's
// total, and one shuffle hands candidate l's total to lane l. Roundings on
// any path: V + 2 + log2 G, inside the bound fast_rho(d, 1) states.
template <int G, int V>
__device__ __forceinline__ void row_slices_g(const float *__restrict__ row, int d4, int lane,
                                             float4 (&f)[V]) {
    const int g = lane % G;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int q = g + G * v;
        f[v] = q < d4 ? __ldg(reinterpret_cast<const float4 *>(row) + q)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int G, int V>
__device__ __forceinline__ float warp_sqdist32g(const float *__restrict__ X, int d,
                                                const float4 (&fx)[V], int fixed, int cand,
                                                int lane) {
    constexpr int R = 32 / G;   // rows per step
    const int d4 = d >> 2, g = lane % G, h = lane / G;
    float acc[G];
#pragma unroll
    for (int s = 0; s < G; ++s) {
        // dead slots read the fixed row (in L1) so every load is unconditional
        const int id = __shfl_sync(0xffffffffu, cand, s * R + h);
        const float4 *row = reinterpret_cast<const float4 *>(X + int64_t(id >= 0 ? id : fixed) * d);
        unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int q = g + G * v;
            if (q < d4) {
                const float4 y = __ldg(row + q);
                a0 = f2_sqacc(f2_sub(f2_pack(y.x, y.y), f2_pack(fx[v].x, fx[v].y)), a0);
                a1 = f2_sqacc(f2_sub(f2_pack(y.z, y.w), f2_pack(fx[v].z, fx[v].w)), a1);
            }
        }
        acc[s] = f2_hsum(f2_add(a0, a1));
    }
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? acc[i] : acc[i + o];
            const float keep = up ? acc[i + o] : acc[i];
            acc[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
    }
    // lane (h, g) holds slot g R + h; slot l sits in lane (l % R) G + l / R
    const float tot = __shfl_sync(0xffffffffu, acc[0], (lane % R) * G + lane / R);
    return cand >= 0 ? tot : 0.0f;
}

// Same layout for 32 independent pairs: lane l holds the pair (a[l], b[l])
// (a < 0: none, result 0) and receives fl-sum of (X[a] - X[b])^2.
template <int G, int V>
__device__ __forceinline__ float warp_pairsq32g(const float *__restrict__ X, int d, int a, int b,
                                                int lane) {
    constexpr int R = 32 / G;
    const int d4 = d >> 2, g = lane % G, h = lane / G;
    float acc[G];
#pragma unroll
    for (int s = 0; s < G; ++s) {
        const int ia = __shfl_sync(0xffffffffu, a, s * R + h);
        const int ib = __shfl_sync(0xffffffffu, b, s * R + h);
        const float4 *ra = reinterpret_cast<const float4 *>(X + int64_t(ia >= 0 ? ia : 0) * d);
        const float4 *rb = reinterpret_cast<const float4 *>(X + int64_t(ia >= 0 ? ib : 0) * d);
        unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int q = g + G * v;
            if (q < d4) {
                const float4 x = __ldg(ra + q), y = __ldg(rb + q);
                a0 = f2_sqacc(f2_sub(f2_pack(x.x, x.y), f2_pack(y.x, y.y)), a0);
                a1 = f2_sqacc(f2_sub(f2_pack(x.z, x.w), f2_pack(y.z, y.w)), a1);
            }
        }
        acc[s] = f2_hsum(f2_add(a0, a1));
    }
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? acc[i] : acc[i + o];
            const float keep = up ? acc[i + o] : acc[i];
            acc[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
    }
    const float tot = __shfl_sync(0xffffffffu, acc[0], (lane % R) * G + lane / R);
    return a >= 0 ? tot : 0.0f;
}

// mma.sync m16n8k16 BF16 -> FP32 (D = A B + C), the warp-level tensor
// instruction; used for 32-candidate dot products where a tcgen05 tile
// would be mostly empty.
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1,
                                               uint32_t a2, uint32_t a3, uint32_t b0,
                                               uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Lanes per row for the grouped sums with V = 4 float4 per lane (0: d too
// large or not a multiple of 4).
inline int sq_group(int d) {
    if (d % 4 != 0) return 0;
    const int need = (d / 4 + 3) / 4;
    int g = 2;
    while (g < need) g <<= 1;
    return g <= 32 ? g : 0;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw; SC'11): ten rounds of
// (c0,c1,c2,c3) <- (hi(B*c2)^c1^k0, lo(B*c2), hi(A*c0)^c3^k1, lo(A*c0)),
// A = 0xD2511F53, B = 0xCD9E8D57, key advanced by (0x9E3779B9, 0xBB67AE85)
// before every round after the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ void set_status(int *dstatus, int bit) {
    atomicOr(dstatus, bit);
}

// ------------------------------------------------ launchers (host side)

// knn_fp32.cu
// Exact kNN of query rows (qrows == nullptr: rows q0..q0+nq-1, written to
// output rows 0..nq-1; else the listed rows, written to their own rows of
// nbr/dist) against all n points, FP32 tiles computing the canonical
// distance. k <= 128.
// colcomp (optional): component of every point; a query's keys in its own
// component are skipped (nearest foreign neighbours).
famst_status knn_fp32(const Exec &ex, Arena &ar, const float *X, int64_t n, int d,
                      int k, const int32_t *qrows, int64_t q0, int64_t nq,
                      int32_t *nbr, float *dist, const int32_t *colcomp = nullptr);
size_t knn_fp32_workspace(int64_t n, int d, int k, int64_t nq, int num_sms);

// Batched launches lay the clouds out in a padded row space: cloud b
// occupies rows roff[b] .. roff[b] + n_b - 1 of a zero-padded copy whose
// clouds start on 256-row boundaries, so a query or key tile never straddles
// two clouds. Compact (unpadded) ids are padded row - shift.
struct TcTile {
    int q0;        // first padded query row of the CTA (128 rows)
    int kt0, kt1;  // the cloud's 256-key tiles [kt0, kt1)
    int nkb;       // active 64-wide K blocks of the hi part
    int row_end;   // padded rows >= row_end are padding
    int shift;     // compact id = padded row - shift
    int part;      // 0: the query tile's whole key list; s > 0: one part of a split
                   // list, whose rows' sorted candidates go to side slot s - 1
};
// Long key lists of a pruned Phase 1 are split so that no work item holds
// much more than a share of one SM's tiles: at most PRUNE_SPLIT_TILES query
// tiles are split, into at most PRUNE_SPLIT_SLOTS parts in all; a list is
// split when longer than max(PRUNE_SPLIT_MIN, visited / PRUNE_SPLIT_TILES).
constexpr int PRUNE_SPLIT_TILES = 640;
constexpr int PRUNE_SPLIT_SLOTS = 2 * PRUNE_SPLIT_TILES;
constexpr int PRUNE_SPLIT_MIN = 16;
struct F32Tile {
    int qbase;     // first query row of the block (64 rows)
    int nq;        // valid queries in the block
    int tile0, tile1;  // key tiles [tile0, tile1) of 128 rows starting at key_base
    int key_base;  // row of key tile 0
    int key_end;   // rows >= key_end are not keys of this cloud
    int d;         // active dimensions of the cloud
    int shift;     // output id = row - shift
};
// Per-cloud description used by the batched re-rank / fallback kernels.
struct CloudDev {
    long long voff;   // first compact id
    int n;            // points
    int d;            // dimensions
    int d_pad;        // tensor-tile K extent (multiple of 64)
    int use_tc;       // 1: rows come from the tensor tiles (re-rank them)
};

// Batched FP32 path: the tiles keep kp = k + 8 candidates per row (c, w,
// N x kp), then canonical re-rank and certificate, then exact rows within
// the cloud for rows it cannot certify (fails / nfail, N + 1 entries).
famst_status knn_fp32_batched(const Exec &ex, const float *Xc, int ld, const long long *voff,
                              int B, const CloudDev *cl, int k, int kp, const F32Tile *tiles,
                              int64_t nblocks, int32_t *c, float *w, int32_t *fails,
                              int32_t *nfail, int32_t *nbr, float *dist);

// knn_tc.cu
// Exact kNN through tcgen05 BF16 (x3 = hi/lo split) distance tiles, FP32
// re-rank, certificate, FP32 recomputation of uncertified rows.
bool knn_tc_supported(int64_t n, int d, int k, bool x3, bool f8 = false);
size_t knn_tc_workspace(int64_t n, int d, int k, bool x3, int num_sms, bool prune = false,
                        bool f8 = false);
// Exact kNN of the listed rows of a batch of clouds (warp per row, canonical
// distances within the row's cloud); rows / count on the device. k <= 64.
famst_status fallback_rows_batched(const Exec &ex, const float *Xc, int ld, const long long *voff,
                                   int B, const CloudDev *cl, int k, const int32_t *rows,
                                   const int32_t *count, int32_t *nbr, float *dist);
famst_status knn_tc(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, int k, bool x3,
                    bool vec4, int32_t *nbr, float *dist, int32_t *pinned_host,
                    int64_t *uncertified, const int32_t *colcomp = nullptr, bool prune = false,
                    int64_t *tiles_visited = nullptr, bool f8 = false);

// prune.cu
// Tile pruning of Phase 1: locality partition (pivot cells), ball bounds,
// per-query-tile lists of the key tiles that may hold a neighbour, and the
// lower bound skip_Q on the distance to every skipped key.
struct PruneOut {
    int32_t *perm = nullptr;        // sorted position -> point
    __nv_bfloat16 *Hs = nullptr;    // operand rows in sorted order
    float *nys = nullptr;           // key norms in sorted order (+inf padding)
    int32_t *klist = nullptr;       // key tiles per query tile
    TcTile *tab = nullptr;          // work items: parts of split lists, then whole lists
    int32_t *nitems = nullptr;      // device: work items in tab (<= nq + PRUNE_SPLIT_SLOTS)
    int32_t *splitq = nullptr;      // device: per split query tile (q, first slot, parts)
    int32_t *nsplit = nullptr;      // device: split query tiles
    float *skipQ = nullptr;         // per query tile
    float *Xs = nullptr;            // the points in sorted order (FP32, n x d)
    float *tau_row = nullptr;       // per sorted row: upper bound on its k-th neighbour distance
    int32_t *visited = nullptr;     // device: number of visited (query, key) tile pairs
    int64_t nq = 0, nk = 0;
};
int prune_pivots(int64_t n);      // evenly spaced pivots
int prune_extra(int64_t n);       // pivots added by each of the two coverage passes
int prune_pivots_max(int64_t n);
bool prune_supported(int64_t n, int d, int k, bool vec4);
size_t prune_workspace(int64_t n, int d, int kh, int kp, int64_t nq, int64_t nk);
famst_status prune_pivot_operands(const Exec &ex, const __nv_bfloat16 *H, int kh, const float *ny,
                                  int64_t n, int K, int Kpad, int32_t *piv, __nv_bfloat16 *Hp,
                                  float *nyp);
// me (host): how many of the M new pivot slots hold distinct far points
// (the others repeat one point); only those need scoring
famst_status prune_augment(const Exec &ex, Arena &ar, const float *xn2, const float *s1, int64_t n,
                           const __nv_bfloat16 *H, int kh, const float *ny, int M, int K,
                           int32_t *piv, __nv_bfloat16 *Hp, float *nyp, int *me);
famst_status prune_partition(const Exec &ex, Arena &ar, const float *X, int d, int64_t n, int k,
                             const __nv_bfloat16 *H, int kh, const float *ny, int nkb, int K,
                             const int32_t *piv, const int32_t *acand, int akp,
                             int32_t *pinned_host, PruneOut *out);


}  // namespace famst
#include <cuda.h>
#include <cuda_bf16.h>
namespace famst {
// Tile shape of the batched tensor pass for operand width D: epi_req = 8
// asks for eight epilogue warps (granted when the lists and three ring
// stages fit), 4 for four; the ring takes what shared memory leaves.
bool knn_tc_batched_plan(int D, int k, bool x3, int epi_req, int *stages, size_t *smem, int *kc,
                         int *epi);
famst_status knn_tc_batched_tiles(const Exec &ex, int D, bool x3, int stages, size_t smem, int kc,
                                  int epi, const TcTile *tiles, int64_t nctas, const float *ny,
                                  int32_t *cand, float *splus, const CUtensorMap *mA,
                                  const CUtensorMap *mB, bool spiral = false);
famst_status knn_tc_batched(const Exec &ex, const float *Xc, int D, int64_t N, int64_t NP,
                            const long long *voff, const long long *roff, int B,
                            const CloudDev *cl, const TcTile *tiles, int64_t nctas, int k,
                            bool x3, int stages, size_t smem, int kc, int epi, __nv_bfloat16 *H,
                            float *ny, float *xn2, float *mean, unsigned *ymax, int32_t *cand,
                            float *splus, int32_t *fail_rows, int32_t *fail_count, int32_t *nbr,
                            float *dist, const CUtensorMap *mA, const CUtensorMap *mB,
                            const float *Xorig = nullptr, const int32_t *perm = nullptr);
bool knn_tc_batched_maps(const void *H, int64_t NP, int D, bool x3, CUtensorMap *mA,
                         CUtensorMap *mB);

// nndescent.cu: Phase 1 by NN-Descent (k <= 32, S <= 32)
bool nndescent_supported(int64_t n, int d, int k, int S);
size_t nndescent_workspace(int64_t n, int d, int k, int S);
famst_status nndescent(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, int k, int S,
                       int max_iters, double delta, uint64_t seed, const int32_t *init,
                       int32_t *nbr, float *dist, int32_t *pinned_host, int32_t *iters_out,
                       int64_t *updates, int64_t *pairs);

// graph.cu
famst_status exclusive_scan_i32(const Exec &ex, Arena &ar, const int32_t *in,
                                int32_t *out, int64_t count, int32_t *total_dev);
size_t scan_workspace(int64_t count);
famst_status radix_sort_pairs(const Exec &ex, Arena &ar, uint32_t *keys, int32_t *vals,
                              int64_t count, int key_bits);
size_t radix_sort_workspace(int64_t count);
famst_status components_uf(const Exec &ex, Arena &ar, const int32_t *nbr, int64_t n,
                           int k, int32_t *comp, int32_t *t_dev);
size_t components_workspace(int64_t n);
famst_status member_lists(const Exec &ex, Arena &ar, const int32_t *comp, int64_t n,
                          int64_t t, int32_t *members, int32_t *comp_off);
size_t member_lists_workspace(int64_t n, int64_t t);
famst_status reverse_csr(const Exec &ex, Arena &ar, const int32_t *nbr, int64_t n, int k,
                         int32_t *rev_off, int32_t *rev_src);
size_t reverse_csr_workspace(int64_t n, int k);

// connect_refine.cu
// BF16 copies of the points for the Alg. 4 filter (see warp_dot32_mma);
// h == nullptr: the filter reads the FP32 rows.
// G[c] of every vertex as one deduplicated list (the kNN list of c, then
// the reverse entries not already in it): entries off[c] .. off[c+1]-1 hold
// the neighbour's id and (eb, ||h||^2) of its BF16 row.
struct GLists {
    const int32_t *off = nullptr;
    const int32_t *id = nullptr;
    const float2 *en = nullptr;
};

struct HalfRows {
    const __nv_bfloat16 *h = nullptr;
    int ld = 0;                  // multiple of 64, zero beyond d
    const float *eb = nullptr;   // per-row error bound
    const float *m = nullptr;    // the centre m (d values)
    const float *n2 = nullptr;   // per row: ||h||^2 (FP32 sum of the exact squares)
    GLists g;   // deduplicated G lists for the staged refinement scans
};
size_t half_rows_workspace(int64_t n, int d);
famst_status half_rows(const Exec &ex, Arena &ar, const float *X, int64_t n, int d,
                       HalfRows *out);
// refine_staged.cu: deduplicated G lists; Algorithm 4 inside a build with
// candidate rows staged in shared memory (sweep-synchronous grouped scans,
// then per-edge fixed points for the last active edges)
size_t glists_workspace(int64_t n, int k);
famst_status refine_glists(const Exec &ex, Arena &ar, const int32_t *nbr, int64_t n, int k,
                           const int32_t *rev_off, const int32_t *rev_src, HalfRows *hr);
bool refine_staged_supported(const HalfRows &hr);
famst_status launch_refine_staged(const Exec &ex, const float *X, int d, const HalfRows &hr,
                                  int32_t *eu, int32_t *ev, float *ew, const int32_t *order,
                                  int64_t m, int max_iters, int32_t *change_hist,
                                  unsigned long long *next_item, unsigned long long *evals);
size_t refine_build_workspace(int64_t n, int64_t m);
famst_status refine_build(const Exec &ex, Arena &ar, const float *X, int d, const HalfRows &hr,
                          const int32_t *members, int64_t n, int32_t *eu, int32_t *ev, float *ew,
                          const int32_t *order, int64_t m, int max_iters, int32_t *change_hist,
                          unsigned long long *evals, int32_t *pinned_host);
// connect_nearest.cu: the lambda nearest pairs of every component pair
size_t connect_nearest_workspace(int64_t n, int64_t t, int lambda);
famst_status connect_nearest(const Exec &ex, Arena &ar, const float *X, int d,
                             const HalfRows &hr, const int32_t *members,
                             const int32_t *comp_off, const int32_t *comp_off_host, int64_t t,
                             int lambda, int32_t *eu, int32_t *ev, float *ew, int32_t *eci,
                             int32_t *ecj, unsigned long long *stats);
// hr (optional): the build's centred BF16 rows; the filter then reads
// those instead of the FP32 rows (same edges)
famst_status connect_edges(const Exec &ex, const float *X, int d, bool vec4,
                           const int32_t *members, const int32_t *comp_off, int64_t t,
                           int lambda, uint64_t seed, int32_t *eu, int32_t *ev, float *ew,
                           int32_t *eci, int32_t *ecj, const HalfRows *hr = nullptr);
famst_status connect_edges_batched(const Exec &ex, const float *X, int ld, int dc,
                                   const int32_t *members, const int32_t *comp_off,
                                   const long long *pp, const int32_t *cbase, int B, int lambda,
                                   uint64_t seed, int64_t m_cap, int32_t *eu, int32_t *ev,
                                   float *ew, int32_t *eci, int32_t *ecj);
famst_status refine_edges(const Exec &ex, Arena &ar, const float *X, int d, bool vec4,
                          const int32_t *nbr, int k, const int32_t *rev_off,
                          const int32_t *rev_src, const int32_t *comp, int64_t t, int32_t *eu,
                          int32_t *ev, float *ew, const int32_t *eci, const int32_t *ecj,
                          int64_t m, int max_iters, int32_t *change_hist /*max_iters+1*/,
                          unsigned long long *evals = nullptr, bool check = true,
                          int *variant = nullptr);
// candidate filter of the refinement kernel that ran (build info)
constexpr int REFINE_FILTER_NONE = 0;      // canonical distance per lane
constexpr int REFINE_FILTER_FP32 = 1;      // FP32 grouped sums + canonical survivors
constexpr int REFINE_FILTER_BF16_MMA = 2;  // BF16 dot products (mma.sync) + canonical survivors
size_t refine_workspace(int64_t m);
famst_status refine_edges_dev(const Exec &ex, Arena &ar, const float *X, int d, bool vec4,
                              const int32_t *nbr, int k, const int32_t *rev_off,
                              const int32_t *rev_src, const int32_t *comp, int32_t *eu,
                              int32_t *ev, float *ew, const int32_t *eci, const int32_t *ecj,
                              int64_t m_cap, const int64_t *m_dev, int max_iters,
                              int32_t *change_hist);

// mst.cu
struct MstOut {
    int32_t *tu, *tv;
    float *tw;
};
// Boruvka state for callers that drive the rounds themselves (exact EMST).
struct BvState {
    int64_t n = 0;
    int round = 0;   // rounds run so far
    // the lists are the exact top-k by (w, id) (their first entry is every
    // vertex's lightest edge): the first round needs no edge scan
    bool knn_exact = false;
    unsigned long long *best1 = nullptr;
    unsigned int *best2 = nullptr;
    int32_t *comp = nullptr;   // component representative of every vertex
    int32_t *newp = nullptr, *flag = nullptr, *pos = nullptr, *rmn = nullptr, *rmx = nullptr;
    float *rw = nullptr;
    int32_t *total = nullptr;
    // compaction (ecap > 0): each scan also writes the edges it found between
    // two components, a superset of the next round's; later rounds read that
    // list (ping-pong, count on the device)
    int64_t ecap = 0;
    int cur = -1;   // list the next round reads; -1: the caller's edges
    int32_t *cu[2] = {nullptr, nullptr}, *cv[2] = {nullptr, nullptr};
    float *cw[2] = {nullptr, nullptr};
    unsigned long long *ccount = nullptr;   // [2]
};
famst_status bv_state_init(const Exec &ex, Arena &ar, int64_t n, BvState *S, int64_t ecap = 0);
famst_status bv_round(const Exec &ex, Arena &ar, BvState &S, const int32_t *nbr, const float *dist,
                      int k, const int32_t *eu, const int32_t *ev, const float *ew, int64_t m,
                      MstOut out, int64_t base, int32_t *added_host);
famst_status boruvka(const Exec &ex, Arena &ar, int64_t n, const int32_t *nbr,
                     const float *dist, int k, const int32_t *eu, const int32_t *ev,
                     const float *ew, int64_t m, MstOut out, int64_t *tree_edges,
                     int *rounds, int32_t *pinned_host, bool knn_exact = false, bool compact = false);
size_t boruvka_workspace(int64_t n, int64_t ecap = 0);
famst_status boruvka_dev(const Exec &ex, Arena &ar, int64_t n, const int32_t *nbr,
                         const float *dist, int k, const int32_t *eu, const int32_t *ev,
                         const float *ew, int64_t m_cap, const int64_t *m_dev, MstOut out,
                         int64_t out_cap, int max_rounds, long long *edges_dev, int *rounds_dev);
famst_status tree_weight(const Exec &ex, Arena &ar, const float *X, int d, bool vec4,
                         const int32_t *tu, const int32_t *tv, const float *tw, int64_t m,
                         double *W_dev /*2 doubles: W, W64*/);
size_t tree_weight_workspace(int64_t m);
famst_status mst_backward(const Exec &ex, Arena &ar, const float *X, int64_t n, int d,
                          bool vec4, const int32_t *tu, const int32_t *tv, int64_t m,
                          float gW, float *gX);
size_t mst_backward_workspace(int64_t n, int64_t m);

// emst.cu
// Exact EMST of the complete graph: Boruvka rounds over masked exact 1-NN
// passes (tc: tensor tiles with precision x3, else FP32 tiles).
size_t emst_workspace(int64_t n, int d, bool tc, bool x3, int num_sms);
famst_status emst_exact(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, bool tc,
                        bool x3, bool vec4, MstOut out, int64_t *tree_edges, int *rounds,
                        int64_t *uncertified, int32_t *pin_knn, int32_t *pin_bv);

// prep (famst_api.cu)
famst_status check_finite(const Exec &ex, const float *X, int64_t count);

}  // namespace famst
