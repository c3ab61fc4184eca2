// Phase 1 by NN-Descent (Dong, Charikar and Li, WWW 2011): the approximate
// kNN graph the paper's Phase 1 takes from an NN-Descent library (Sec. 2,
// Sec. 3 "GetANNs"), for clouds where the exact n^2 d tiles cost too much.
//
// Every step is defined on sets, so the result does not depend on the order
// in which the GPU makes its comparisons, and equals the CPU restatement bit
// for bit:
//   lists    B[v]: k distinct ids, (w, id) ascending, a "new" flag each;
//   start    the first k distinct of the draws u = pick(r0, n-1) (u += 1 if
//            u >= v), r0 of Philox4x32-10(counter (v, r, 0, 1)), r < 8k,
//            then the smallest unused ids; all new;
//   sample   per v and class (new / old): the S candidates smallest in
//            (pr, u) among the ids of that class in B[v] and the ids u
//            whose B[u] holds v with that class, pr = r0 of Philox(counter
//            (v, u, it, 2)); sampled new entries of B[v] become old;
//   join     every pair {a, b} (a, b in new[v], or a in new[v] and b in
//            old[v], a != b) proposes b to B[a] and a to B[b] at w(a, b);
//   update   B[a] = the k smallest distinct (w, id) of B[a] and its
//            proposals, entries from proposals new; c = entries added;
//   stop     after an iteration with c = 0 or c < delta n k.
//
// GPU layout: a list is k 64-bit keys (w bits << 32 | id) plus a flag byte
// per entry, one warp per list (lane r = entry r). The join stages a v's
// (at most 2S) candidate rows in shared memory and gives every thread one
// pair: the canonical FP32 distance with its 32 partials in registers,
// float4 reads of the shared rows (row stride an odd number of 16-byte
// units, so the rows that 8 neighbouring lanes read sit in different bank
// groups). A proposal is kept only if it beats the target's current k-th
// key: the k-th key of a list only falls while proposals arrive, so this
// drops nothing the update would keep. The joins of a chunk of v's append
// their proposals to one buffer; the buffer is grouped by target (count,
// scan, scatter) and each target's warp merges its proposals into its list
// (sort the batch, bitonic merge with the list, duplicates dropped) before
// the next chunk joins.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "famst_internal.cuh"

namespace famst {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint8_t NND_NEW = 1, NND_INS = 2;
constexpr uint32_t TAG_START = 1, TAG_PRIO = 2;
constexpr int NND_JOIN_THREADS = 128;

__device__ __forceinline__ uint32_t nnd_draw(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             uint2 key) {
    return philox4x32_10(make_uint4(c0, c1, c2, c3), key).x;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Bitonic sort of one key per lane, ascending by lane, moving a payload
// with its key. Equal keys are never exchanged.
__device__ __forceinline__ void warp_sort_asc(uint64_t &k, uint32_t &p, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t ok = shfl_xor_u64(k, stride);
            const uint32_t op = __shfl_xor_sync(FULL, p, stride);
            const bool up = (lane & size) == 0 || size == 32;
            const bool lower = (lane & stride) == 0;
            const bool take = (lower == up) ? (ok < k) : (ok > k);
            if (take) {
                k = ok;
                p = op;
            }
        }
    }
}

// Sort a bitonic sequence (one key per lane) ascending.
__device__ __forceinline__ void warp_bitonic_merge_asc(uint64_t &k, uint32_t &p, int lane) {
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        const uint64_t ok = shfl_xor_u64(k, stride);
        const uint32_t op = __shfl_xor_sync(FULL, p, stride);
        const bool lower = (lane & stride) == 0;
        const bool take = lower ? (ok < k) : (ok > k);
        if (take) {
            k = ok;
            p = op;
        }
    }
}

// L (sorted ascending, KEY_NONE beyond its entries) <- the 32 smallest of L
// and the batch b (unsorted, KEY_NONE = empty), payloads moving with keys.
__device__ __forceinline__ void warp_merge_batch(uint64_t &L, uint32_t &Lp, uint64_t b,
                                                 uint32_t bp, int lane) {
    warp_sort_asc(b, bp, lane);
    const uint64_t rb = shfl_idx_u64(b, 31 - lane);
    const uint32_t rbp = __shfl_sync(FULL, bp, 31 - lane);
    if (rb < L) {
        L = rb;
        Lp = rbp;
    }
    warp_bitonic_merge_asc(L, Lp, lane);
}

// Lanes [have, have + popc(keep)) below k receive the kept values of the
// lanes in `keep`, in lane order, through the warp's 32-slot scratch.
__device__ __forceinline__ int compact_into(int acc, int u, bool kept, int have, int k,
                                            volatile int *scratch, int lane) {
    const unsigned keep = __ballot_sync(FULL, kept);
    const int rank = __popc(keep & lanemask_lt());
    if (kept && have + rank < k) scratch[have + rank] = u;
    __syncwarp();
    const int got = __popc(keep);
    if (lane >= have && lane < have + got && lane < k) acc = scratch[lane];
    __syncwarp();
    return acc;
}

// Start lists: one warp per v.
__global__ void nnd_start_kernel(const float *__restrict__ X, int n, int d, int k, uint2 key,
                                 const int32_t *__restrict__ init, uint64_t *__restrict__ Bk,
                                 uint8_t *__restrict__ Bf, int *dstatus) {
    __shared__ int scratch[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int v = blockIdx.x * (blockDim.x >> 5) + wib;
    if (v >= n) return;
    volatile int *sc = scratch[wib];
    int acc = -1, have = 0;
    if (init) {
        if (lane < k) acc = __ldg(init + int64_t(v) * k + lane);
        const unsigned same = __match_any_sync(FULL, acc);
        const bool bad = lane < k && (acc < 0 || acc >= n || acc == v ||
                                      (same & lanemask_lt()) != 0);
        if (__any_sync(FULL, bad)) {
            if (lane == 0) set_status(dstatus, STATUS_BAD_ID);
            return;
        }
        have = k;
    }
    for (int base = 0; base < 8 * k && have < k; base += 32) {
        const int r = base + lane;
        int u = -1;
        if (r < 8 * k) {
            u = int((uint64_t(nnd_draw(uint32_t(v), uint32_t(r), 0u, TAG_START, key)) *
                     uint64_t(n - 1)) >> 32);
            if (u >= v) ++u;
        }
        bool dup = u < 0;
        for (int q = 0; q < have; ++q) dup |= __shfl_sync(FULL, acc, q) == u;
        dup |= (__match_any_sync(FULL, u) & lanemask_lt()) != 0;   // an earlier draw
        acc = compact_into(acc, u, !dup, have, k, sc, lane);
        have = min(k, have + __popc(__ballot_sync(FULL, !dup)));
    }
    for (int base = 0; have < k && base < n; base += 32) {   // n - 1 >= k ids to fill from
        const int u = base + lane;
        bool dup = u >= n || u == v;
        for (int q = 0; q < have; ++q) dup |= __shfl_sync(FULL, acc, q) == u;
        acc = compact_into(acc, u, !dup, have, k, sc, lane);
        have = min(k, have + __popc(__ballot_sync(FULL, !dup)));
    }
    float w = 0.0f;
    const float *xv = X + int64_t(v) * d;
    for (int r = 0; r < k; ++r) {
        const int id = __shfl_sync(FULL, acc, r);
        const float wr = __fsqrt_rn(canon_p_warp(xv, X + int64_t(id) * d, d, lane));
        if (lane == r) w = wr;
    }
    uint64_t kk = lane < k ? nb_key(w, uint32_t(acc)) : KEY_NONE;
    uint32_t dummy = 0;
    warp_sort_asc(kk, dummy, lane);
    if (lane < k) {
        Bk[int64_t(v) * k + lane] = kk;
        Bf[int64_t(v) * k + lane] = NND_NEW;
    }
}

// Reverse entries of each class: row cls * n + u lists the v with u in B[v].
__global__ void nnd_rev_count_kernel(const uint64_t *__restrict__ Bk,
                                     const uint8_t *__restrict__ Bf, int64_t nk, int n,
                                     int32_t *__restrict__ cnt) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nk) return;
    const int u = int(key_lo(Bk[e]));
    const int cls = (Bf[e] & NND_NEW) ? 0 : 1;
    atomicAdd(cnt + int64_t(cls) * n + u, 1);
}

__global__ void nnd_rev_scatter_kernel(const uint64_t *__restrict__ Bk,
                                       const uint8_t *__restrict__ Bf, int64_t nk, int n, int k,
                                       const int32_t *__restrict__ off, int32_t *__restrict__ cnt,
                                       int32_t *__restrict__ src) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nk) return;
    const int u = int(key_lo(Bk[e]));
    const int64_t row = int64_t((Bf[e] & NND_NEW) ? 0 : 1) * n + u;
    const int pos = off[row] + atomicSub(cnt + row, 1) - 1;   // leaves cnt at 0
    src[pos] = int32_t(e / k);
}

// Samples new[v], old[v] (S ids each, -1 beyond the count) and the flag
// update of step 2. One warp per v.
__global__ void nnd_sample_kernel(const uint64_t *__restrict__ Bk, uint8_t *__restrict__ Bf,
                                  int n, int k, int S, int it, uint2 key,
                                  const int32_t *__restrict__ off,
                                  const int32_t *__restrict__ src, int32_t *__restrict__ samp,
                                  int32_t *__restrict__ scnt) {
    const int lane = threadIdx.x & 31;
    const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (v >= n) return;
    const uint64_t ek = lane < k ? Bk[int64_t(v) * k + lane] : KEY_NONE;
    const uint8_t fl0 = lane < k ? Bf[int64_t(v) * k + lane] : uint8_t(0);
    uint8_t fl = fl0;   // classes come from the flags as the iteration found them
    const uint32_t id = key_lo(ek);
    uint32_t dummy = 0;
    for (int cls = 0; cls < 2; ++cls) {
        const bool mine = lane < k && ((fl0 & NND_NEW) != 0) == (cls == 0);
        const uint64_t fk =
            mine ? (uint64_t(nnd_draw(uint32_t(v), id, uint32_t(it), TAG_PRIO, key)) << 32) | id
                 : KEY_NONE;
        uint64_t L = fk;
        warp_sort_asc(L, dummy, lane);
        if (lane >= S) L = KEY_NONE;
        const int64_t row = int64_t(cls) * n + v;
        const int r0 = off[row], r1 = off[row + 1];
        for (int b = r0; b < r1; b += 32) {
            const int q = b + lane;
            uint64_t c = KEY_NONE;
            if (q < r1) {
                const uint32_t u = uint32_t(src[q]);
                c = (uint64_t(nnd_draw(uint32_t(v), u, uint32_t(it), TAG_PRIO, key)) << 32) | u;
            }
            // an id in both directions is one candidate (same key)
            for (int r = 0; r < k; ++r)
                if (shfl_idx_u64(fk, r) == c) c = KEY_NONE;
            if (c >= shfl_idx_u64(L, S - 1)) c = KEY_NONE;
            if (__all_sync(FULL, c == KEY_NONE)) continue;
            warp_merge_batch(L, dummy, c, 0u, lane);
            if (lane >= S) L = KEY_NONE;
        }
        const unsigned has = __ballot_sync(FULL, L != KEY_NONE);
        if (lane < S) samp[row * S + lane] = L != KEY_NONE ? int32_t(uint32_t(L)) : -1;
        if (lane == 0) scnt[row] = __popc(has);
        if (cls == 0) {
            bool hit = false;
            for (int q = 0; q < S; ++q) {
                const uint64_t lq = shfl_idx_u64(L, q);
                hit |= fk != KEY_NONE && lq == fk;
            }
            if (hit) fl &= uint8_t(~NND_NEW);
        }
    }
    if (lane < k) Bf[int64_t(v) * k + lane] = fl;
}

// Local joins of v in [v0, v0 + gridDim.x): one block per v.
__global__ void __launch_bounds__(NND_JOIN_THREADS)
nnd_join_kernel(const float *__restrict__ X, int d, int n, int k, int S, int v0, int rs4,
                const int32_t *__restrict__ samp, const int32_t *__restrict__ scnt,
                const uint64_t *__restrict__ Bk, int32_t *__restrict__ pt,
                uint64_t *__restrict__ pk, unsigned long long *__restrict__ pcount,
                unsigned long long pcap, unsigned long long *__restrict__ npairs, int vec4,
                int *dstatus) {
    extern __shared__ float4 srow[];
    __shared__ int sid[64];
    __shared__ unsigned long long sthr[64];
    __shared__ unsigned spairs;
    const int v = v0 + blockIdx.x;
    const int nn = scnt[v], no = scnt[n + v];
    const int m = nn + no;
    if (nn == 0) return;   // every pair holds a new candidate
    if (threadIdx.x == 0) spairs = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int id = i < nn ? samp[int64_t(v) * S + i] : samp[(int64_t(n) + v) * S + i - nn];
        sid[i] = id;
        sthr[i] = Bk[int64_t(id) * k + k - 1];
    }
    __syncthreads();
    if (vec4) {   // rows 16-byte aligned, d % 4 == 0: one float4 per load
        const int d4v = d >> 2;
        for (int e = threadIdx.x; e < m * rs4; e += blockDim.x) {
            const int r = e / rs4, c4 = e - r * rs4;
            srow[e] = c4 < d4v ? __ldg(reinterpret_cast<const float4 *>(X + int64_t(sid[r]) * d) + c4)
                               : make_float4(0.f, 0.f, 0.f, 0.f);   // zeros add nothing
        }
    } else {
        float *sf = reinterpret_cast<float *>(srow);
        const int dp = rs4 * 4;
        for (int e = threadIdx.x; e < m * dp; e += blockDim.x) {
            const int r = e / dp, t = e - r * dp;
            sf[e] = t < d ? __ldg(X + int64_t(sid[r]) * d + t) : 0.0f;   // zeros add nothing
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int d4 = (d + 3) >> 2;
    unsigned my_pairs = 0;
    for (int i = warp; i < nn; i += nw) {
        const int ia = sid[i];
        const uint64_t ta = sthr[i];
        const float4 *ra = srow + i * rs4;
        for (int b0 = i + 1; b0 < m; b0 += 32) {
            const int b = b0 + lane;
            const bool live = b < m && sid[b < m ? b : i] != ia;
            my_pairs += __popc(__ballot_sync(FULL, live));
            float p[32];
#pragma unroll
            for (int l = 0; l < 32; ++l) p[l] = 0.0f;
            if (live) {
                const float4 *rb = srow + b * rs4;
                for (int q0 = 0; q0 < d4; q0 += 8) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (q0 + j < d4) {
                            const float4 x = ra[q0 + j], y = rb[q0 + j];
                            const float t0 = __fsub_rn(x.x, y.x), t1 = __fsub_rn(x.y, y.y);
                            const float t2 = __fsub_rn(x.z, y.z), t3 = __fsub_rn(x.w, y.w);
                            p[4 * j + 0] = __fmaf_rn(t0, t0, p[4 * j + 0]);
                            p[4 * j + 1] = __fmaf_rn(t1, t1, p[4 * j + 1]);
                            p[4 * j + 2] = __fmaf_rn(t2, t2, p[4 * j + 2]);
                            p[4 * j + 3] = __fmaf_rn(t3, t3, p[4 * j + 3]);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
                for (int l = 0; l < o; ++l) p[l] = __fadd_rn(p[l], p[l + o]);
            }
            const float w = __fsqrt_rn(p[0]);
            const int ib = live ? sid[b] : 0;
            const bool to_a = live && nb_key(w, uint32_t(ib)) < ta;
            const bool to_b = live && nb_key(w, uint32_t(ia)) < sthr[live ? b : 0];
            const unsigned ma = __ballot_sync(FULL, to_a), mb = __ballot_sync(FULL, to_b);
            const int tot = __popc(ma) + __popc(mb);
            if (tot == 0) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(pcount, (unsigned long long)tot);
            base = __shfl_sync(FULL, base, 0);
            if (base + tot > pcap) {   // the chunk size rules this out
                if (lane == 0) set_status(dstatus, STATUS_INTERNAL);
                continue;
            }
            if (to_a) {
                const unsigned long long q = base + __popc(ma & lanemask_lt());
                pt[q] = ia;
                pk[q] = nb_key(w, uint32_t(ib));
            }
            if (to_b) {
                const unsigned long long q = base + __popc(ma) + __popc(mb & lanemask_lt());
                pt[q] = ib;
                pk[q] = nb_key(w, uint32_t(ia));
            }
        }
    }
    if (lane == 0 && my_pairs) atomicAdd(&spairs, my_pairs);
    __syncthreads();
    if (threadIdx.x == 0 && spairs) atomicAdd(npairs, (unsigned long long)spairs);
}

// proposals per target; the targets that receive any are listed once each
// (in no particular order: each target's merge is independent)
__global__ void nnd_group_count_kernel(const int32_t *__restrict__ pt,
                                       const unsigned long long *__restrict__ pcount,
                                       unsigned long long pcap, int32_t *__restrict__ gcnt,
                                       int32_t *__restrict__ act, int32_t *__restrict__ nact) {
    const unsigned long long np = *pcount < pcap ? *pcount : pcap;
    for (unsigned long long q = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < np;
         q += uint64_t(gridDim.x) * blockDim.x) {
        const int t = pt[q];
        if (atomicAdd(gcnt + t, 1) == 0) act[atomicAdd(nact, 1)] = t;
    }
}

__global__ void nnd_group_scatter_kernel(const int32_t *__restrict__ pt,
                                         const uint64_t *__restrict__ pk,
                                         const unsigned long long *__restrict__ pcount,
                                         unsigned long long pcap,
                                         const int32_t *__restrict__ goff,
                                         int32_t *__restrict__ gcnt, uint64_t *__restrict__ gk) {
    const unsigned long long np = *pcount < pcap ? *pcount : pcap;
    for (unsigned long long q = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < np;
         q += uint64_t(gridDim.x) * blockDim.x) {
        const int t = pt[q];
        const int pos = goff[t] + atomicSub(gcnt + t, 1) - 1;   // leaves gcnt at 0
        gk[pos] = pk[q];
    }
}

// B[a] <- the k smallest distinct keys of B[a] and a's grouped proposals,
// for the listed targets a (one warp per target, the warps striding over the
// list).
__global__ void nnd_merge_kernel(int k, const int32_t *__restrict__ act,
                                 const int32_t *__restrict__ nact, const int32_t *__restrict__ goff,
                                 const uint64_t *__restrict__ gk, uint64_t *__restrict__ Bk,
                                 uint8_t *__restrict__ Bf) {
    const int lane = threadIdx.x & 31;
    const int na = *nact;
    const int nwarps = int(gridDim.x * (blockDim.x >> 5));
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < na; w += nwarps) {
    const int a = act[w];
    const int g0 = goff[a], g1 = goff[a + 1];
    uint64_t L = lane < k ? Bk[int64_t(a) * k + lane] : KEY_NONE;
    uint32_t Lf = lane < k ? Bf[int64_t(a) * k + lane] : 0u;
    bool changed = false;
    for (int b = g0; b < g1; b += 32) {
        uint64_t c = b + lane < g1 ? gk[b + lane] : KEY_NONE;
        if (c >= shfl_idx_u64(L, k - 1)) c = KEY_NONE;
        // an id already in the list has the same key: keep the entry
        const uint32_t cid = key_lo(c);
        for (int r = 0; r < k; ++r) {
            const uint32_t lr = __shfl_sync(FULL, key_lo(L), r);
            if (c != KEY_NONE && lr == cid) c = KEY_NONE;
        }
        // the same proposal from several joins: keep one
        if ((__match_any_sync(FULL, c) & lanemask_lt()) != 0) c = KEY_NONE;
        if (__all_sync(FULL, c == KEY_NONE)) continue;
        warp_merge_batch(L, Lf, c, uint32_t(NND_NEW | NND_INS), lane);
        if (lane >= k) L = KEY_NONE;
        changed = true;
    }
    if (changed && lane < k) {
        Bk[int64_t(a) * k + lane] = L;
        Bf[int64_t(a) * k + lane] = uint8_t(Lf);
    }
    }
}

__global__ void nnd_count_inserted_kernel(uint8_t *__restrict__ Bf, int64_t nk,
                                          unsigned long long *__restrict__ c) {
    unsigned long long mine = 0;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nk;
         e += int64_t(gridDim.x) * blockDim.x) {
        const uint8_t f = Bf[e];
        if (f & NND_INS) {
            ++mine;
            Bf[e] = uint8_t(f & ~NND_INS);
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(c, mine);
}

__global__ void nnd_output_kernel(const uint64_t *__restrict__ Bk, int64_t nk,
                                  int32_t *__restrict__ nbr, float *__restrict__ dist) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nk) return;
    const uint64_t kk = Bk[e];
    nbr[e] = int32_t(key_lo(kk));
    dist[e] = key_w(kk);
}

struct NndPlan {
    int rs4;          // shared row stride in float4 units (odd)
    size_t smem;      // join kernel dynamic shared memory
    int64_t pcap;     // proposal buffer entries
    int64_t chunk;    // v per join launch
};

NndPlan nnd_plan(int64_t n, int d, int S) {
    NndPlan p{};
    p.rs4 = ((d + 3) / 4) | 1;
    p.smem = size_t(2 * S) * p.rs4 * 16;
    const int64_t per_v = int64_t(S) * (3 * S - 1);   // 2 proposals per pair
    p.pcap = std::min<int64_t>(std::max<int64_t>(per_v, int64_t(1) << 28), n * per_v);
    p.chunk = std::max<int64_t>(1, p.pcap / per_v);
    return p;
}

}  // namespace

bool nndescent_supported(int64_t n, int d, int k, int S) {
    if (n < 2 || k < 1 || k > 32 || k > n - 1 || S < 1 || S > 32 || d < 1) return false;
    if (n * int64_t(k) >= (int64_t(1) << 31)) return false;
    return nnd_plan(n, d, S).smem <= 200 * 1024;
}

size_t nndescent_workspace(int64_t n, int d, int k, int S) {
    const NndPlan p = nnd_plan(n, d, S);
    size_t b = 0;
    b += align256(size_t(n) * k * 8) + align256(size_t(n) * k);     // keys, flags
    b += align256(size_t(2) * n * S * 4) + align256(size_t(2) * n * 4);   // samples
    b += align256(size_t(2 * n + 1) * 4) * 2 + align256(size_t(n) * k * 4);   // reverse
    b += align256(size_t(n + 1) * 4) * 2;                            // group counts, offsets
    b += align256(size_t(n) * 4) + 256;                              // active targets
    b += align256(size_t(p.pcap) * 4) + align256(size_t(p.pcap) * 8) * 2;
    b += 256 * 4;
    b += scan_workspace(2 * n + 1);
    return b;
}

famst_status nndescent(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, int k, int S,
                       int max_iters, double delta, uint64_t seed, const int32_t *init,
                       int32_t *nbr, float *dist, int32_t *pinned_host, int32_t *iters_out,
                       int64_t *updates, int64_t *pairs) {
    if (!nndescent_supported(n, d, k, S)) return FAMST_ERR_UNSUPPORTED;
    const NndPlan P = nnd_plan(n, d, S);
    const int64_t nk = n * k;
    uint64_t *Bk = ar.take<uint64_t>(size_t(nk));
    uint8_t *Bf = ar.take<uint8_t>(size_t(nk));
    int32_t *samp = ar.take<int32_t>(size_t(2) * n * S);
    int32_t *scnt = ar.take<int32_t>(size_t(2) * n);
    int32_t *rcnt = ar.take<int32_t>(size_t(2 * n + 1));
    int32_t *roff = ar.take<int32_t>(size_t(2 * n + 1));
    int32_t *rsrc = ar.take<int32_t>(size_t(nk));
    int32_t *gcnt = ar.take<int32_t>(size_t(n + 1));
    int32_t *goff = ar.take<int32_t>(size_t(n + 1));
    int32_t *act = ar.take<int32_t>(size_t(n));     // targets with proposals in a chunk
    int32_t *nact = ar.take<int32_t>(1);
    int32_t *pt = ar.take<int32_t>(size_t(P.pcap));
    uint64_t *pk = ar.take<uint64_t>(size_t(P.pcap));
    uint64_t *gk = ar.take<uint64_t>(size_t(P.pcap));
    unsigned long long *pcount = ar.take<unsigned long long>(1);
    unsigned long long *cdev = ar.take<unsigned long long>(2);   // c, pairs
    if (!Bk || !Bf || !samp || !scnt || !rcnt || !roff || !rsrc || !gcnt || !goff || !pt ||
        !pk || !gk || !pcount || !cdev || !act || !nact)
        return FAMST_ERR_OOM;
    const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
    const int ni = int(n);
    const bool vec4 = (d % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
    const unsigned wgrid = unsigned((n + 7) / 8);   // 8 warps per block
    const unsigned egrid = unsigned((nk + 255) / 256);
    const unsigned sgrid = unsigned(ex.num_sms) * 8;
    FAMST_LAUNCH(ex, nnd_start_kernel, wgrid, 256, 0, X, ni, d, k, key, init, Bk, Bf,
                 ex.dstatus);
    if (init) {   // a bad start list stops here, before any list is read
        if (cudaMemcpyAsync(pinned_host, ex.dstatus, 4, cudaMemcpyDeviceToHost, ex.stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        if (pinned_host[0] & STATUS_BAD_ID) return FAMST_ERR_INVALID_ARG;
    }
    if (cudaMemsetAsync(rcnt, 0, size_t(2 * n + 1) * 4, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(gcnt, 0, size_t(n + 1) * 4, ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    if (set_smem_attr(nnd_join_kernel, P.smem, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    int it = 0;
    while (it < max_iters) {
        if (cudaMemsetAsync(cdev, 0, 16, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
        // step 1: reverse entries by class, samples; step 2 inside
        FAMST_LAUNCH(ex, nnd_rev_count_kernel, egrid, 256, 0, Bk, Bf, nk, ni, rcnt);
        // the scans' block sums are scratch: the arena returns to its mark
        const size_t mark = ar.off;
        famst_status st = exclusive_scan_i32(ex, ar, rcnt, roff, 2 * n + 1, nullptr);
        ar.off = mark;
        if (st != FAMST_OK) return st;
        FAMST_LAUNCH(ex, nnd_rev_scatter_kernel, egrid, 256, 0, Bk, Bf, nk, ni, k, roff, rcnt,
                     rsrc);
        FAMST_LAUNCH(ex, nnd_sample_kernel, wgrid, 256, 0, Bk, Bf, ni, k, S, it, key, roff, rsrc,
                     samp, scnt);
        // steps 3 and 4, chunk by chunk
        for (int64_t v0 = 0; v0 < n; v0 += P.chunk) {
            const int64_t nv = std::min<int64_t>(P.chunk, n - v0);
            if (cudaMemsetAsync(pcount, 0, 8, ex.stream) != cudaSuccess ||
                cudaMemsetAsync(nact, 0, 4, ex.stream) != cudaSuccess)
                return FAMST_ERR_CUDA;
            FAMST_LAUNCH(ex, nnd_join_kernel, unsigned(nv), NND_JOIN_THREADS, P.smem, X, d, ni, k,
                         S, int(v0), P.rs4, samp, scnt, Bk, pt, pk, pcount,
                         (unsigned long long)P.pcap, cdev + 1, int(vec4), ex.dstatus);
            FAMST_LAUNCH(ex, nnd_group_count_kernel, sgrid, 256, 0, pt, pcount,
                         (unsigned long long)P.pcap, gcnt, act, nact);
            st = exclusive_scan_i32(ex, ar, gcnt, goff, n + 1, nullptr);
            ar.off = mark;
            if (st != FAMST_OK) return st;
            FAMST_LAUNCH(ex, nnd_group_scatter_kernel, sgrid, 256, 0, pt, pk, pcount,
                         (unsigned long long)P.pcap, goff, gcnt, gk);
            FAMST_LAUNCH(ex, nnd_merge_kernel, sgrid, 256, 0, k, act, nact, goff, gk, Bk, Bf);
        }
        FAMST_LAUNCH(ex, nnd_count_inserted_kernel, sgrid, 256, 0, Bf, nk, cdev);
        if (cudaMemcpyAsync(pinned_host, cdev, 16, cudaMemcpyDeviceToHost, ex.stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(pinned_host + 4, ex.dstatus, 4, cudaMemcpyDeviceToHost, ex.stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        if (pinned_host[4] & STATUS_INTERNAL) return FAMST_ERR_CUDA;
        int64_t c = 0, np = 0;
        std::memcpy(&c, pinned_host, 8);
        std::memcpy(&np, pinned_host + 2, 8);
        if (updates) updates[it] = c;
        if (pairs) pairs[it] = np;
        ++it;
        if (c == 0 || double(c) < delta * double(n) * double(k)) break;
    }
    FAMST_LAUNCH(ex, nnd_output_kernel, egrid, 256, 0, Bk, nk, nbr, dist);
    if (iters_out) *iters_out = it;
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst
