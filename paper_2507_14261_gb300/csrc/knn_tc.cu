// Phase 1 (Algorithm 1, GetANNs) on tcgen05 tensor cores, exact result.
//
// Score. With centred coordinates x' = fl(x - mean), the squared distance
// is ||x'_i||^2 + s(i,j) with s(i,j) = ||x'_j||^2 - 2 x'_i . x'_j; the first
// term is constant along a row, so rows are ranked by s. The dot products
// run on the tensor cores in BF16 with FP32 accumulation: BF16 mode uses
// xh = bf16(x'); BF16X3 mode adds the two correction products of the
// hi/lo split x' ~ xh + xl (xh.yh + xl.yh + xh.yl), whose error is
// O(2^-16) instead of O(2^-8).
//
// Kernel (one CTA per 128 query rows, 64 + 32 E threads, E = 8 or 4):
//   warp 0     TMA producer: the query tile's operand rows once (resident),
//              then 256-key tiles, one 64-wide K block per ring stage;
//   warp 1     allocates 512 TMEM columns (two 128 x 256 FP32
//              accumulators) and one lane issues tcgen05.mma (M=128, N=256,
//              K=16 per instruction) with SW128 K-major smem descriptors;
//              tcgen05.commit frees ring stages and publishes accumulators;
//   warps 2..  E epilogue warps: thread r of a warp owns query row r of its
//              TMEM lane quarter; with E = 8 two warps share a quarter, each
//              on half of the columns. It loads 16 columns at a time with
//              tcgen05.ld, forms s = ny_j - 2 acc (key norms read from L1),
//              and stages the columns that beat its row's threshold in
//              shared memory. When any lane's stage is nearly full the warp
//              merges the stages, eight candidates at a time (a sorting
//              network, then a bitonic merge: topk_merge.cuh), into per-row
//              sorted register lists of the KC smallest scores, then
//              tightens the threshold to the KC-th score (the smaller of the
//              two halves' when E = 8); the halves' lists merge at the end.
// Work items: a query tile with its key tiles (all of them, or a pruned
// list); a long pruned list is split into parts run by separate CTAs, whose
// rows' lists split_merge_kernel combines.
// Nothing of the n x n score matrix leaves the SM. Every mbarrier wait is
// bounded in time; on expiry the CTA sets an error bit, drains its own
// copies and MMAs, frees its TMEM and returns.
//
// Exactness. Row i keeps k' = KC-1 candidates and s+ = its KC-th smallest
// score. The rerank kernel computes the canonical FP32 distance of every
// candidate, takes the k smallest (w, id), and certifies the row when a
// rigorous bound on the score error proves that no unkept point can have a
// canonical distance <= the k-th. Uncertified rows are recomputed by the
// FP32 SIMT tiles, so the output equals the exact brute-force kNN.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "famst_internal.cuh"
#include "mbarrier.cuh"
#include "topk_merge.cuh"

namespace famst {
namespace {

constexpr int BM = 128;          // query rows per CTA (TMEM lanes)
constexpr int BN = 256;          // keys per tile (accumulator columns)
constexpr int BK = 64;           // K elements per stage (one 128-byte swizzle atom)
constexpr int A_BLOCK = BM * BK * 2;   // 16 KB
constexpr int B_BLOCK = BN * BK * 2;   // 32 KB
constexpr int CAPB = 24;         // staged candidates per row (flush check every 16 columns)
constexpr int TC_THREADS_MAX = 64 + 32 * 8;   // producer, MMA issuer, up to 8 epilogue warps

// ------------------------------------------------------------ PTX helpers

// Bounded wait for the phase of parity `parity` to complete. Returns false
// if the CTA aborted or the time limit expired (then it raises the abort).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            set_status(status, STATUS_LOOP_LIMIT);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 inputs, FP32 accumulate)
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on `bar` once every tcgen05 op issued so far by this thread is done
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}
__device__ __forceinline__ void epilogue_bar(int nthreads) {  // the epilogue warps only
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
// The same barrier, returning whether any epilogue thread passed p = true.
__device__ __forceinline__ bool epilogue_bar_any(int nthreads, bool p) {
    int r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.s32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, 1, %2, pi;\n\tselp.s32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"(int(p)), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// of 128 bytes, 8-row groups 1024 bytes apart (SBO), version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);   // start address
    d |= uint64_t(1) << 16;                    // leading byte offset (unused with SW128 K-major)
    d |= uint64_t(1024 >> 4) << 32;            // stride byte offset
    d |= uint64_t(1) << 46;                    // descriptor version
    d |= uint64_t(2) << 61;                    // SWIZZLE_128B
    return d;
}
// Instruction descriptor, kind::f16: D F32, A/B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) |
           (uint32_t(M >> 4) << 24);
}

// Instruction descriptor, kind::f8f6f4: D F32, A/B E4M3 (format 0), both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f8f6f4 (E4M3 inputs, FP32 accumulate;
// K = 32 per instruction, 32 bytes of each K-major row as for kind::f16)
__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

struct TcArgs {
    int n;
    int nk_tiles;
    int nkb;        // 64-wide K blocks of the hi part (d_pad / 64)
    int x3;         // hi/lo split on
    int stages;     // B ring depth
    const float *ny;    // key norms ||x'_j||^2, +inf beyond n (nk_tiles * BN entries)
    int32_t *cand;      // n x (KC - 1)
    float *splus;       // n
    int *status;
    const TcTile *tiles;  // null: one cloud, CTA b = query tile b over all keys
    const int32_t *colcomp;  // MASK: component of every (padded) row; pairs in one component are skipped
    const int32_t *klist;    // non-null: CTA key tiles are klist[kt0 .. kt1) instead of kt0 .. kt1
    int cross;               // queries and keys are different sets: no self-exclusion
    int epi;                 // epilogue warps: 8 (two per TMEM lane quarter, each on half
                             // of the columns) or 4 (0 reads as 4)
    const float *rscale;     // FP8 operands: per-row scale s (x' ~ s q), query and key rows
                             // alike (keys padded with 1 to nk_tiles * BN entries)
    const float *thr0;       // non-null: per query row, a score every one of its k nearest
                             // keys stays below (the lists start there; s+ is capped by it)
    int nitems;              // > 0: work items (query tiles) handed to the CTAs round-robin
                             // (persistent launch, grid <= nitems); 0: one per CTA
    int spiral;              // 1: an item's key tiles [kt0, kt1) are visited outward from the
                             // query tile's own (q0 / BN, then +1, -1, +2, ...): on rows in
                             // a spatial order the lists fill with near keys first
    const int32_t *nitems_dev;  // non-null (one item per CTA): CTAs from *nitems_dev on are idle
    int32_t *side_j;         // items that are parts of a split list (TcTile::part = s + 1):
    float *side_s;           //   per slot s and tile row, the KC - 1 smallest (id, score),
    float *side_splus;       //   ascending, and the part's s+
};

template <int KC>
__device__ __forceinline__ void list_insert(float (&ls)[KC], int (&lj)[KC], float s, int j) {
    // (s, j) goes before the first entry greater than s; the entries from
    // there on move one place up. Every slot is computed from the old
    // ls[p - 1], ls[p] and s alone (no value carried from slot to slot), so
    // the KC updates are independent instructions rather than one chain.
#pragma unroll
    for (int p = KC - 1; p >= 1; --p) {
        const bool up = ls[p - 1] > s;   // the entry below moves here
        const bool here = ls[p] > s;
        ls[p] = up ? ls[p - 1] : (here ? s : ls[p]);
        lj[p] = up ? lj[p - 1] : (here ? j : lj[p]);
    }
    const bool here0 = ls[0] > s;
    ls[0] = here0 ? s : ls[0];
    lj[0] = here0 ? j : lj[0];
}

template <int KC, bool MASK, bool F8 = false>
__global__ void __launch_bounds__(KC <= 2 * CAPB ? TC_THREADS_MAX : 64 + 32 * 4, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              TcArgs args) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzle atoms
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // Work items: query tile `item` with its key tiles. A CTA takes items
    // blockIdx.x, blockIdx.x + gridDim.x, ...; TMEM, barriers and the
    // pipeline state carry over from one item to the next.
    // a launch sized for the most items a table can hold: the CTAs beyond
    // the table's count leave before touching barriers or TMEM
    if (args.nitems_dev && int(blockIdx.x) >= __ldg(args.nitems_dev)) return;
    const int nitems = args.nitems > 0 ? args.nitems : int(gridDim.x);
    struct Item {
        int q0, kt0, kt1, nkb, row_end, shift, part;
    };
    auto item_of = [&](int item) {
        Item I;
        if (args.tiles) {
            const TcTile T = args.tiles[item];
            I.q0 = T.q0; I.kt0 = T.kt0; I.kt1 = T.kt1; I.nkb = T.nkb; I.row_end = T.row_end;
            I.shift = T.shift;
            I.part = T.part;
        } else {
            I.q0 = item * BM; I.kt0 = 0; I.kt1 = args.nk_tiles; I.nkb = args.nkb;
            I.row_end = args.n; I.shift = 0; I.part = 0;
        }
        return I;
    };
    // key tile of the t-th step of an item
    auto ktile = [&](const Item &I, int t) {
        if (args.klist) return __ldg(args.klist + I.kt0 + t);
        if (!args.spiral) return I.kt0 + t;
        const int c0 = min(max(I.q0 / BN, I.kt0), I.kt1 - 1);
        const int L = c0 - I.kt0, R = I.kt1 - 1 - c0, m = min(L, R);
        if (t <= 2 * m) return (t & 1) ? c0 + ((t + 1) >> 1) : c0 - (t >> 1);
        return R > L ? c0 + (t - m) : c0 - (t - m);
    };
    const int nA_max = (args.x3 ? 2 : 1) * args.nkb;  // resident A blocks (widest item)
    unsigned char *sA = base;
    unsigned char *sB = sA + size_t(nA_max) * A_BLOCK;
    const int EPI = args.epi == 8 ? 8 : 4;
    const int NH = EPI / 4;                           // column halves (1 or 2)
    // staging [NH][CAPB][BM] scores and ids; with two halves, the second
    // half's final list ([KC][BM], KC <= 2 CAPB) reuses it for the merge
    float *stg_s = reinterpret_cast<float *>(sB + size_t(args.stages) * B_BLOCK);
    int *stg_j = reinterpret_cast<int *>(stg_s + NH * CAPB * BM);
    volatile float *thr_sh = reinterpret_cast<volatile float *>(stg_j + NH * CAPB * BM);  // [2][BM]
    uint64_t *bars = reinterpret_cast<uint64_t *>(
        reinterpret_cast<unsigned char *>(stg_j + NH * CAPB * BM) + 2 * BM * 4);
    uint64_t *full = bars;                       // [stages]
    uint64_t *empty = bars + args.stages;        // [stages]
    uint64_t *a_full = bars + 2 * args.stages;
    uint64_t *tfull = a_full + 1;                // [2]
    uint64_t *tempty = tfull + 2;                // [2]
    uint64_t *mma_done = tempty + 2;
    uint64_t *a_empty = mma_done + 1;            // the A blocks may be overwritten
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(a_empty + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < args.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI);
        }
        mbar_init(mma_done, 1);
        mbar_init(a_empty, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    for (int x = threadIdx.x; x < 2 * BM; x += blockDim.x) thr_sh[x] = __int_as_float(0x7f800000);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA))
                         : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB))
                         : "memory");
            int it = 0, a_issued = 0;   // B blocks and A batches issued
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const Item I = item_of(item);
                // the previous item's MMAs must be done with the A blocks
                if (a_issued > 0 && !mbar_wait(a_empty, (a_issued - 1) & 1, abort_flag,
                                               args.status)) {
                    ok = false;
                    break;
                }
                const int nA = (args.x3 ? 2 : 1) * I.nkb;
                mbar_expect_tx(a_full, uint32_t(nA) * A_BLOCK);
                // resident A blocks: hi blocks 0..nkb-1, then lo blocks (at column
                // block args.nkb + kb of the operand rows)
                for (int a = 0; a < nA; ++a) {
                    const int col = a < I.nkb ? a : args.nkb + (a - I.nkb);
                    tma_load_2d(sA + size_t(a) * A_BLOCK, &tmA, a_full, col * (F8 ? 2 * BK : BK),
                                I.q0);
                }
                ++a_issued;
                const int nkb_tile = args.x3 ? 2 * I.nkb : I.nkb;   // B blocks per key tile
                const int total = (I.kt1 - I.kt0) * nkb_tile;
                for (int j = 0; j < total; ++j, ++it) {
                    const int s = it % args.stages, r = it / args.stages;
                    if (!mbar_wait(&empty[s], (r & 1) ^ 1, abort_flag, args.status)) {
                        ok = false;
                        break;
                    }
                    const int t = ktile(I, j / nkb_tile), blk = j % nkb_tile;
                    // x3 order per key tile: hi_0, lo_0, hi_1, lo_1, ...
                    const int col =
                        args.x3 ? ((blk & 1) ? args.nkb + (blk >> 1) : (blk >> 1)) : blk;
                    mbar_expect_tx(&full[s], B_BLOCK);
                    tma_load_2d(sB + size_t(s) * B_BLOCK, &tmB, &full[s],
                                col * (F8 ? 2 * BK : BK), t * BN);
                }
            }
            // drain: every issued copy must land before the CTA leaves
            if (a_issued > 0) mbar_drain(a_full, (a_issued - 1) & 1);
            for (int s = 0; s < args.stages && s < it; ++s) {
                int last = s + ((it - 1 - s) / args.stages) * args.stages;  // last use of stage s
                mbar_drain(&full[s], (last / args.stages) & 1);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = F8 ? idesc_e4m3(BM, BN) : idesc_bf16(BM, BN);
            int it = 0, g = 0, na = 0;   // B blocks, key tiles and items consumed
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++na) {
                const Item I = item_of(item);
                if (!mbar_wait(a_full, na & 1, abort_flag, args.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int ntiles = I.kt1 - I.kt0;
                const int nkb_tile = args.x3 ? 2 * I.nkb : I.nkb;
                for (int t = 0; t < ntiles && ok; ++t, ++g) {
                    const int b = g & 1, use = g >> 1;
                    if (!mbar_wait(&tempty[b], (use & 1) ^ 1, abort_flag, args.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + uint32_t(b * BN);
                    uint32_t acc = 0;
                    for (int blk = 0; blk < nkb_tile; ++blk, ++it) {
                        const int s = it % args.stages, r = it / args.stages;
                        if (!mbar_wait(&full[s], r & 1, abort_flag, args.status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t bsm = smem_u32(sB + size_t(s) * B_BLOCK);
                        const int kb = args.x3 ? (blk >> 1) : blk;
                        const bool is_lo = args.x3 && (blk & 1);
                        // which resident A blocks multiply this B block
                        const int nq = args.x3 ? (is_lo ? 1 : 2) : 1;
                        for (int q = 0; q < nq; ++q) {
                            // hi B block: A_hi then A_lo; lo B block: A_hi
                            const int ablk = (q == 0) ? kb : I.nkb + kb;
                            const uint32_t asm_ = smem_u32(sA + size_t(ablk) * A_BLOCK);
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                if constexpr (F8)
                                    umma_f8(d_tmem, sdesc_sw128(asm_ + kk * 32),
                                            sdesc_sw128(bsm + kk * 32), IDESC, acc);
                                else
                                    umma_f16(d_tmem, sdesc_sw128(asm_ + kk * 32),
                                             sdesc_sw128(bsm + kk * 32), IDESC, acc);
                                acc = 1;
                            }
                        }
                        umma_commit(&empty[s]);  // stage s is free once these MMAs finish
                    }
                    if (!ok) break;
                    umma_commit(&tfull[b]);      // accumulator b is complete
                }
                if (!ok) break;
                umma_commit(a_empty);            // this item's A blocks are free once done
            }
            umma_commit(mma_done);
            mbar_drain(mma_done, 0);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue
        const int quarter = warp & 3;               // TMEM lanes 32*quarter ..
        const int half = (warp - 2) >> 2;           // columns [half * ncols, + ncols)
        const int ncols = BN / NH;
        const int col0 = half * ncols;
        const int row = quarter * 32 + lane;
        float *my_s = stg_s + half * CAPB * BM + row;
        int *my_j = stg_j + half * CAPB * BM + row;
        int g = 0;   // key tiles consumed (accumulator buffer g & 1)
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const Item I = item_of(item);
        const int i = I.q0 + row;
        const int ntiles = I.kt1 - I.kt0;
        float ls[KC];
        int lj[KC];
#pragma unroll
        for (int p = 0; p < KC; ++p) {
            ls[p] = __int_as_float(0x7f800000);
            lj[p] = -1;
        }
        const float thr0v = (args.thr0 && i < args.n) ? __ldg(args.thr0 + i)
                                                      : __int_as_float(0x7f800000);
        float thr = thr0v;
        int cnt = 0;
        // With two halves each list sees half the columns. A score at or above
        // the other list's KC-th is not in the row's KC smallest (that list
        // alone holds KC scores below it), so both filter with the smaller
        // of the two thresholds.
        auto partner_thr = [&]() {
            return NH == 2 ? thr_sh[(1 - half) * BM + row] : __int_as_float(0x7f800000);
        };
        auto flush = [&]() {
            const int mx = __reduce_max_sync(0xffffffffu, cnt);
            const float pt = partner_thr();
            if constexpr (KC >= 32) {
                // eight staged candidates at a time: those still below the
                // list's KC-th score are sorted and merged into the list
                for (int q0 = 0; q0 < mx; q0 += 8) {
                    const float lim = fminf(ls[KC - 1], pt);
                    float bs[8];
                    int bj[8];
                    int nq = 0;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float sv = __int_as_float(0x7f800000);
                        int jv = -1;
                        if (q0 + c < cnt) {
                            const float s = my_s[(q0 + c) * BM];
                            const int j = my_j[(q0 + c) * BM];
                            if ((args.cross || j != i) && s < lim) {
                                sv = s;
                                jv = j;
                                ++nq;
                            }
                        }
                        bs[c] = sv;
                        bj[c] = jv;
                    }
                    // one merging network for any number of entries: a
                    // single-insertion shortcut beside it measured slower
                    // (instruction-fetch stalls from the larger loop body)
                    if (__reduce_max_sync(0xffffffffu, nq) == 0) continue;
                    topk::sort8(bs, bj);
                    topk::merge8<KC>(ls, lj, bs, bj);
                }
            } else {
                for (int q = 0; q < mx; ++q) {
                    if (q < cnt) {
                        float sv = my_s[q * BM];
                        int jv = my_j[q * BM];
                        if ((args.cross || jv != i) && sv < fminf(ls[KC - 1], pt))
                            list_insert<KC>(ls, lj, sv, jv);
                    }
                }
            }
            cnt = 0;
            if (NH == 2) thr_sh[half * BM + row] = ls[KC - 1];
            thr = fminf(fminf(ls[KC - 1], pt), thr0v);
        };
        bool ok = true;
        int my_comp = 0;
        if constexpr (MASK) my_comp = __ldg(args.colcomp + i);
        // FP8: acc = q_i . q_j, so x'_i . x'_j ~ s_i s_j acc
        float m2s = -2.0f;
        if constexpr (F8) m2s = -2.0f * (i < args.n ? __ldg(args.rscale + i) : 1.0f);
        for (int t = 0; t < ntiles; ++t, ++g) {
            const int b = g & 1, use = g >> 1;
            // every lane waits; the warp proceeds only if all lanes saw the phase
            const bool got = mbar_wait(&tfull[b], use & 1, abort_flag, args.status);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t tb =
                tmem + (uint32_t(quarter * 32) << 16) + uint32_t(b * BN + col0);
            const int kt_this = ktile(I, t);
            // key norms (and components) of this tile's columns straight from
            // global memory: every lane reads the same addresses (L1 broadcast);
            // the next tile's are prefetched into L1 meanwhile
            const float *nyt = args.ny + size_t(kt_this) * BN + col0;
            const int *cmt = MASK ? args.colcomp + size_t(kt_this) * BN + col0 : nullptr;
            if (t + 1 < ntiles && lane < ncols / 32) {
                const size_t nxt = size_t(ktile(I, t + 1)) * BN + col0 + 32 * lane;
                asm volatile("prefetch.global.L1 [%0];" ::"l"(args.ny + nxt));
                if constexpr (MASK) asm volatile("prefetch.global.L1 [%0];" ::"l"(args.colcomp + nxt));
            }
            thr = fminf(thr, partner_thr());
            // Candidate staging for 16 columns. The divergent part only touches
            // this lane's stage; the warp-collective flush check sits at a
            // warp-uniform point after it.
            auto process = [&](uint32_t(&v)[16], int ch) {
                float mn = __int_as_float(0x7f800000);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const float4 nn = __ldg(reinterpret_cast<const float4 *>(nyt + ch * 16 + 4 * c4));
                    float4 cs = make_float4(m2s, m2s, m2s, m2s);
                    if constexpr (F8) {   // per-key scales, same layout as the norms
                        const float4 sk = __ldg(reinterpret_cast<const float4 *>(
                            args.rscale + (nyt - args.ny) + ch * 16 + 4 * c4));
                        cs = make_float4(m2s * sk.x, m2s * sk.y, m2s * sk.z, m2s * sk.w);
                    }
                    float s0 = fmaf(cs.x, __uint_as_float(v[4 * c4 + 0]), nn.x);
                    float s1 = fmaf(cs.y, __uint_as_float(v[4 * c4 + 1]), nn.y);
                    float s2 = fmaf(cs.z, __uint_as_float(v[4 * c4 + 2]), nn.z);
                    float s3 = fmaf(cs.w, __uint_as_float(v[4 * c4 + 3]), nn.w);
                    if constexpr (MASK) {  // same component: not a candidate
                        const int4 cc = __ldg(reinterpret_cast<const int4 *>(cmt + ch * 16 + 4 * c4));
                        const float inf = __int_as_float(0x7f800000);
                        s0 = cc.x == my_comp ? inf : s0;
                        s1 = cc.y == my_comp ? inf : s1;
                        s2 = cc.z == my_comp ? inf : s2;
                        s3 = cc.w == my_comp ? inf : s3;
                    }
                    v[4 * c4 + 0] = __float_as_uint(s0);
                    v[4 * c4 + 1] = __float_as_uint(s1);
                    v[4 * c4 + 2] = __float_as_uint(s2);
                    v[4 * c4 + 3] = __float_as_uint(s3);
                    mn = fminf(mn, fminf(fminf(s0, s1), fminf(s2, s3)));
                }
                const int j0 = kt_this * BN + col0 + ch * 16;
                if (mn < thr) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        float sc = __uint_as_float(v[c]);
                        if (sc < thr) {
                            my_s[cnt * BM] = sc;
                            my_j[cnt * BM] = j0 + c;
                            ++cnt;
                        }
                    }
                }
                // at most 16 more per chunk: flush before a stage could overflow
                if (__any_sync(0xffffffffu, cnt > CAPB - 16)) flush();
            };
            // two 16-column register buffers: the load of chunk c+1 overlaps the
            // processing of chunk c
            const int nch = ncols / 16;
            uint32_t va[16], vb[16];
            __syncwarp();
            tmem_ld16(tb, va);
#pragma unroll 1
            for (int ch = 0; ch < nch; ch += 2) {
                tmem_ld_wait16(va);
                __syncwarp();
                tmem_ld16(tb + (ch + 1) * 16, vb);
                process(va, ch);
                tmem_ld_wait16(vb);
                __syncwarp();
                if (ch + 2 < nch) tmem_ld16(tb + (ch + 2) * 16, va);
                process(vb, ch + 1);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        flush();
        if (NH == 2) {
            // merge: the second half's list goes through shared memory into the
            // first half's (every epilogue warp reaches both barriers, on the
            // error path too)
            epilogue_bar(32 * EPI);
            if (half == 1) {
#pragma unroll
                for (int p = 0; p < KC; ++p) {
                    stg_s[p * BM + row] = ls[p];
                    stg_j[p * BM + row] = lj[p];
                }
            }
            epilogue_bar(32 * EPI);
            if (half == 0) {
                if constexpr (KC >= 32) {
                    // the other list is ascending: batches of eight, until no
                    // lane has an entry below its KC-th score
                    for (int p0 = 0; p0 < KC; p0 += 8) {
                        const float lim = ls[KC - 1];
                        float bs[8];
                        int bj[8];
                        int nq = 0;
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float s = stg_s[(p0 + c) * BM + row];
                            const bool in = s < lim;
                            bs[c] = in ? s : __int_as_float(0x7f800000);
                            bj[c] = in ? stg_j[(p0 + c) * BM + row] : -1;
                            nq += in;
                        }
                        if (__reduce_max_sync(0xffffffffu, nq) == 0) break;
                        topk::merge8<KC>(ls, lj, bs, bj);
                    }
                } else {
                    for (int p = 0; p < KC; ++p) {   // ascending: stop at the first that cannot enter
                        const float sv = stg_s[p * BM + row];
                        if (!(sv < ls[KC - 1])) break;
                        list_insert<KC>(ls, lj, sv, stg_j[p * BM + row]);
                    }
                }
            }
        }
        if (ok && half == 0 && i < I.row_end) {
            if constexpr (KC == 1) {   // top-1 mode: the best key and its score
                args.cand[i - I.shift] = lj[0] >= 0 ? lj[0] - I.shift : -1;
            } else if (I.part > 0) {   // one part of a split list: scores too, for the merge
                const size_t at = size_t(I.part - 1) * BM + row;
                int32_t *oj = args.side_j + at * (KC - 1);
                float *os = args.side_s + at * (KC - 1);
#pragma unroll
                for (int p = 0; p < KC - 1; ++p) {
                    oj[p] = lj[p] >= 0 ? lj[p] - I.shift : -1;
                    os[p] = ls[p];
                }
                args.side_splus[at] = fminf(ls[KC - 1], thr0v);
            } else {
                int32_t *out = args.cand + size_t(i - I.shift) * (KC - 1);
#pragma unroll
                for (int p = 0; p < KC - 1; ++p) out[p] = lj[p] >= 0 ? lj[p] - I.shift : -1;
            }
            // keys that never entered the list scored at least min(KC-th, thr0)
            if (KC == 1 || I.part == 0) args.splus[i - I.shift] = fminf(ls[KC - 1], thr0v);
        }
        // next item: this row's published threshold starts over, and the
        // staging area is free again; a failure anywhere stops every warp here
        if (NH == 2) thr_sh[half * BM + row] = __int_as_float(0x7f800000);
        if (epilogue_bar_any(32 * EPI, !ok)) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Rows of split query tiles (one block of BM threads per split tile): the
// row's candidates are the KC - 1 smallest scores over its parts' lists and
// s+ = min(the KC-th smallest of those lists, every part's s+). A key that
// no part kept scored at least its part's s+; a kept key left out here
// scored at least the KC-th. So the row gets the candidates and s+ the
// unsplit list would have had (up to the order of equal scores).
template <int KC>
__global__ void __launch_bounds__(BM)
split_merge_kernel(const int32_t *__restrict__ splitq, const int32_t *__restrict__ nsplit,
                   const int32_t *__restrict__ side_j, const float *__restrict__ side_s,
                   const float *__restrict__ side_splus, int64_t n, int32_t *__restrict__ cand,
                   float *__restrict__ splus) {
    if (int(blockIdx.x) >= __ldg(nsplit)) return;
    const int q = splitq[3 * blockIdx.x], slot0 = splitq[3 * blockIdx.x + 1];
    const int P = splitq[3 * blockIdx.x + 2];
    const int row = threadIdx.x;
    const int64_t i = int64_t(q) * BM + row;
    if (i >= n) return;
    float ls[KC];
    int lj[KC];
#pragma unroll
    for (int p = 0; p < KC; ++p) {
        ls[p] = __int_as_float(0x7f800000);
        lj[p] = -1;
    }
    float sp = __int_as_float(0x7f800000);
    for (int part = 0; part < P; ++part) {
        const size_t at = size_t(slot0 + part) * BM + row;
        sp = fminf(sp, side_splus[at]);
        const float *ps = side_s + at * (KC - 1);
        const int32_t *pj = side_j + at * (KC - 1);
        for (int p = 0; p < KC - 1; ++p) {   // ascending: stop at the first that cannot enter
            const float sv = ps[p];
            if (!(sv < ls[KC - 1])) break;
            list_insert<KC>(ls, lj, sv, pj[p]);
        }
    }
    int32_t *out = cand + i * (KC - 1);
#pragma unroll
    for (int p = 0; p < KC - 1; ++p) out[p] = lj[p];
    splus[i] = fminf(ls[KC - 1], sp);
}

// ------------------------------------------------------------- prep

// per-block column sums (double) over a contiguous range of rows
// (the rows in order, eight loads in flight per thread)
__global__ void colsum_partial_kernel(const float *__restrict__ X, int64_t n, int d, int rows_per,
                                      double *__restrict__ part) {
    int64_t r0 = int64_t(blockIdx.x) * rows_per;
    int64_t r1 = r0 + rows_per < n ? r0 + rows_per : n;
    // FP32 sums within the block's rows (the FP64 pipe is slow on this GPU,
    // and the centre only has to be some fixed point near the data: every
    // bound downstream holds for any centre), FP64 across blocks
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        float s = 0.0f;
        int64_t r = r0;
        for (; r + 8 <= r1; r += 8) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __ldg(X + (r + q) * d + c);
#pragma unroll
            for (int q = 0; q < 8; ++q) s += v[q];
        }
        for (; r < r1; ++r) s += __ldg(X + r * d + c);
        part[int64_t(blockIdx.x) * d + c] = double(s);
    }
}

// one block per column: strided partial sums, then a tree in shared memory
__global__ void colsum_final_kernel(const double *__restrict__ part, int nb, int d, int64_t n,
                                    float *__restrict__ mean) {
    __shared__ double red[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) s += part[int64_t(b) * d + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
        if (int(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[c] = float(red[0] / double(n));
}

// One warp per row: centred row, BF16 hi (and lo) operand rows, FP32 norm.
__global__ void tc_prep_kernel(const float *__restrict__ X, int64_t n, int d, int d_pad, int x3,
                               const float *__restrict__ mean, __nv_bfloat16 *__restrict__ H,
                               float *__restrict__ ny, float *__restrict__ xnorm,
                               unsigned *__restrict__ ymax_bits) {
    __shared__ unsigned bmax;
    if (threadIdx.x == 0) bmax = 0u;
    __syncthreads();
    const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row < n) {
        const int kh = (x3 ? 2 : 1) * d_pad;
        __nv_bfloat16 *h = H + row * kh;
        const float *x = X + row * d;
        float acc = 0.0f;
        // four coordinates per lane per step (16-byte rows), else one
        const bool v4 = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
        if (v4) {
            for (int t = 4 * lane; t < d_pad; t += 128) {
                float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t < d) {
                    const float4 a = __ldg(reinterpret_cast<const float4 *>(x + t));
                    const float4 m = __ldg(reinterpret_cast<const float4 *>(mean + t));
                    xv = make_float4(__fsub_rn(a.x, m.x), __fsub_rn(a.y, m.y), __fsub_rn(a.z, m.z),
                                     __fsub_rn(a.w, m.w));
                }
                const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
                __nv_bfloat16 hi[4], lo[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    hi[q] = __float2bfloat16_rn(xs[q]);
                    lo[q] = __float2bfloat16_rn(__fsub_rn(xs[q], __bfloat162float(hi[q])));
                    acc = fmaf(xs[q], xs[q], acc);
                }
                *reinterpret_cast<uint2 *>(h + t) = *reinterpret_cast<const uint2 *>(hi);
                if (x3) *reinterpret_cast<uint2 *>(h + d_pad + t) = *reinterpret_cast<const uint2 *>(lo);
            }
        } else {
            for (int t = lane; t < d_pad; t += 32) {
                float xc = t < d ? __fsub_rn(x[t], mean[t]) : 0.0f;
                __nv_bfloat16 hi = __float2bfloat16_rn(xc);
                h[t] = hi;
                if (x3) h[d_pad + t] = __float2bfloat16_rn(__fsub_rn(xc, __bfloat162float(hi)));
                acc = fmaf(xc, xc, acc);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            ny[row] = acc;
            xnorm[row] = acc;
            atomicMax(&bmax, __float_as_uint(sqrtf(acc)));   // one global atomic per block
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bmax != 0u) atomicMax(ymax_bits, bmax);
}

// One warp per row, FP8 operands: centred row x' = fl(x - mean), scale
// s = 2^e with e the smallest integer such that max |x'| <= 448 s (the
// largest finite E4M3), q = e4m3(x' / s) rounded to nearest (the division by
// a power of two is exact), FP32 norm ||x'||^2 as for the BF16 operands.
// Rows of d_pad bytes, zero beyond d.
__global__ void tc_prep_f8_kernel(const float *__restrict__ X, int64_t n, int d, int d_pad,
                                  const float *__restrict__ mean, uint8_t *__restrict__ Q,
                                  float *__restrict__ rscale, float *__restrict__ ny,
                                  float *__restrict__ xnorm, unsigned *__restrict__ ymax_bits) {
    __shared__ unsigned bmax;
    if (threadIdx.x == 0) bmax = 0u;
    __syncthreads();
    const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row < n) {
        const float *x = X + row * d;
        float amax = 0.0f, acc = 0.0f;
        for (int t = lane; t < d; t += 32) {
            const float xc = __fsub_rn(__ldg(x + t), __ldg(mean + t));
            amax = fmaxf(amax, fabsf(xc));
            acc = fmaf(xc, xc, acc);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
        // smallest e with amax <= 448 2^e (so 2^e < 2 amax / 448), kept to
        // normal FP32 scales; the quotient's rounding is corrected by the
        // exact comparisons with 448 2^e
        int e = 0;
        if (amax > 0.0f) {
            frexpf(amax / 448.0f, &e);   // amax / 448 = f 2^e, 0.5 <= f < 1
            while (e > -126 && ldexpf(448.0f, e - 1) >= amax) e -= 1;
            while (e < 127 && ldexpf(448.0f, e) < amax) e += 1;
        }
        const float sc = ldexpf(1.0f, e);
        uint8_t *q = Q + row * d_pad;
        for (int t = lane; t < d_pad; t += 32) {
            const float xc = t < d ? __fsub_rn(__ldg(x + t), __ldg(mean + t)) : 0.0f;
            q[t] = uint8_t(__nv_cvt_float_to_fp8(ldexpf(xc, -e), __NV_SATFINITE, __NV_E4M3));
        }
        if (lane == 0) {
            rscale[row] = sc;
            ny[row] = acc;
            xnorm[row] = acc;
            atomicMax(&bmax, __float_as_uint(sqrtf(acc)));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bmax != 0u) atomicMax(ymax_bits, bmax);
}

__global__ void fill_value_kernel(float *p, int64_t from, int64_t to, float v) {
    int64_t i = from + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < to) p[i] = v;
}

__global__ void fill_inf_kernel(float *p, int64_t from, int64_t to) {
    int64_t i = from + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < to) p[i] = __int_as_float(0x7f800000);
}

// Start threshold of the pruned tiles' lists: every key y within tau_r of
// row r (tau_r bounds r's k-th neighbour distance from above) has a tile
// score s~(y) = ||y'||^2 - 2 x'.y' (rounded) with s~ <= ||x' - y'||^2 -
// ||x'||^2 + E <= (tau_r + c)^2 - xn2 (1 - (d+1) u) + E, where c bounds the
// centring rounding and E the tile's score error (the certificate's terms).
// Written over tau_row in place.
__global__ void thr0_kernel(float *__restrict__ tau_row, const float *__restrict__ xn2s,
                            int64_t n, int d, const unsigned *__restrict__ ymax_bits,
                            double eps_dot) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double u24 = 1.0 / 16777216.0;
    const double xn2 = double(xn2s[r]), xn = sqrt(xn2);
    const double ym = double(__uint_as_float(*ymax_bits));
    const double E = 2.0 * eps_dot * xn * ym * 1.01 + (d + 1) * u24 * 1.02 * ym * ym +
                     2.0 * u24 * (ym * ym + 2.0 * xn * ym) * 1.01 + 1e-30;
    const double t = (double(tau_row[r]) + 1.02 * u24 * (xn + ym)) * (1.0 + 0x1p-20);
    const double thr = t * t - xn2 * (1.0 - (d + 1) * u24 * 1.02) + E;
    tau_row[r] = __double2float_ru(thr + (thr >= 0.0 ? thr : -thr) * 0x1p-20 + 1e-30);
}

// ------------------------------------------------------------- rerank

struct CertConst {
    double eps_dot;   // relative error of the tensor-core dot (products + accumulation)
    double d_plus;    // d + 4, for the canonical distance error
};

// One warp per row: canonical distances of the k' candidates, bitonic sort
// of (w, id), top k, certificate. Row i's point is xi; candidate ids index
// rows of X (row stride ld, chain length dc >= d: columns beyond d are zero
// and leave the canonical distance unchanged). d is the true dimension used in
// the error bounds. Returns whether the row was certified (then the k
// results are written).
// XR > 0 (dc <= 32 XR): lane l takes coordinates l, l + 32, ... (its
// canonical partial) of every candidate from coalesced row reads, the query
// row held in registers, and the warp sums the partials of a batch of
// candidates at once (below); XR = 0: one candidate per lane, its 32
// partials in registers.
template <int VEC, int KC, int XR = 0>
__device__ __forceinline__ bool rerank_row(const float *__restrict__ X, int ld, int dc, int d,
                                           const float *__restrict__ xi, int k,
                                           const int32_t *__restrict__ cand_row, float sp,
                                           float skip, float xn2f, float ymf, double eps_dot,
                                           int lane,
                                           int32_t *__restrict__ nbr_row,
                                           float *__restrict__ dist_row,
                                           const int32_t *__restrict__ idmap = nullptr) {
    constexpr int KP = KC - 1;
    uint64_t key[2];
    if constexpr (XR > 0) {
        // batches of NB candidates: lane l's partial of candidate c in
        // acc[c mod NB]; the butterfly's steps xor 16 .. xor NB on all NB,
        // then its later steps (xor NB/2 .. 1) transposed, each lane passing
        // on the half it does not keep. The additions are the butterfly's
        // own (same pairs, same order), so lane l ends with the canonical
        // total of candidate NB b + (l mod NB), with 2 NB - 1 + NB log2(32/NB)
        // shuffles per batch instead of 5 NB.
        // (wider rows take smaller batches, within the sorted kernel's
        // register budget; NB = 1 is the plain butterfly)
        constexpr int NB = XR <= 4 ? 16 : (XR <= 8 ? 2 : 1);
        constexpr int G = XR <= 8 ? 2 : 1;   // candidates with loads in flight
        static_assert(NB % G == 0, "a batch is whole load groups");
        float xr[XR];
#pragma unroll
        for (int q = 0; q < XR; ++q) {
            const int t = lane + 32 * q;
            xr[q] = t < dc ? __ldg(xi + t) : 0.0f;
        }
        int jc[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = h * 32 + lane;
            jc[h] = c < KP ? cand_row[c] : -1;
        }
        key[0] = key[1] = KEY_NONE;
#pragma unroll 1
        for (int b = 0; b < (KP + NB - 1) / NB; ++b) {
            float acc[NB];
#pragma unroll
            for (int g0 = 0; g0 < NB; g0 += G) {
                int j[G];
                float y[G][XR];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int c = NB * b + g0 + g;
                    const int ja = __shfl_sync(0xffffffffu, jc[0], c & 31);
                    const int jb = __shfl_sync(0xffffffffu, jc[1], c & 31);
                    j[g] = c < KP ? (c < 32 ? ja : jb) : -1;
#pragma unroll
                    for (int q = 0; q < XR; ++q) {
                        const int t = lane + 32 * q;
                        y[g][q] = (j[g] >= 0 && t < dc) ? __ldg(X + int64_t(j[g]) * ld + t) : 0.0f;
                    }
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float p = 0.0f;
#pragma unroll
                    for (int q = 0; q < XR; ++q) {
                        const float dl = __fsub_rn(xr[q], y[g][q]);
                        p = __fmaf_rn(dl, dl, p);
                    }
                    acc[g0 + g] = p;
                }
            }
#pragma unroll
            for (int o = 16; o >= NB; o >>= 1)
#pragma unroll
                for (int i = 0; i < NB; ++i)
                    acc[i] = __fadd_rn(acc[i], __shfl_xor_sync(0xffffffffu, acc[i], o));
#pragma unroll
            for (int o = NB / 2; o >= 1; o >>= 1) {
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < o; ++i) {
                    const float send = up ? acc[i] : acc[i + o];
                    const float keep = up ? acc[i + o] : acc[i];
                    acc[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
                }
            }
            // candidate c of this lane; sort element c (register c / 32 of
            // lane c mod 32) takes it from the lane of the matching block
            const int c = NB * b + (lane & (NB - 1));
            const int ja = __shfl_sync(0xffffffffu, jc[0], c & 31);
            const int jb = __shfl_sync(0xffffffffu, jc[1], c & 31);
            const int jl = c < KP ? (c < 32 ? ja : jb) : -1;
            if ((lane & ~(NB - 1)) == ((NB * b) & 31) && jl >= 0) {
                const uint64_t kg = nb_key(__fsqrt_rn(acc[0]), uint32_t(idmap ? idmap[jl] : jl));
                if (c < 32) key[0] = kg;
                else key[1] = kg;
            }
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int c = h * 32 + lane;
            key[h] = KEY_NONE;
            if (c < KP) {
                int j = cand_row[c];
                if (j >= 0)
                    key[h] = nb_key(canon_dist<VEC>(xi, X + int64_t(j) * ld, dc),
                                    uint32_t(idmap ? idmap[j] : j));
            }
        }
    }
    // bitonic sort of 64 keys, element index = h*32 + lane
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride == 32) {
                // partner is the other register of the same lane (size == 64: ascending)
                uint64_t lo = key[0] < key[1] ? key[0] : key[1];
                uint64_t hi = key[0] < key[1] ? key[1] : key[0];
                key[0] = lo;
                key[1] = hi;
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int idx = h * 32 + lane;
                    bool asc = ((idx & size) == 0);
                    uint64_t other = shfl_xor_u64(key[h], stride);
                    bool lower = (lane & stride) == 0;
                    uint64_t mn = key[h] < other ? key[h] : other;
                    uint64_t mx = key[h] < other ? other : key[h];
                    key[h] = (lower == asc) ? mn : mx;
                }
            }
        }
    }
    // k-th key (index k-1)
    const int kh = (k - 1) >> 5, kl = (k - 1) & 31;
    uint64_t kth = __shfl_sync(0xffffffffu, kh ? key[1] : key[0], kl);
    bool cert = false;
    if (lane == 0) {
        const double u24c = 1.0 / 16777216.0;
        // keys of skipped tiles lie at true distance >= skip; their canonical
        // distance is then above the k-th when skip (1 - eps_canon) is
        const bool skip_ok = !(skip < __int_as_float(0x7f800000)) ||
                             double(skip) * (1.0 - (d + 4.0) * u24c * 1.05) > double(key_w(kth));
        if (!skip_ok) {
            cert = false;
        } else if (!(sp < __int_as_float(0x7f800000))) {
            cert = true;  // fewer than KC points besides i among the visited keys: all kept
        } else {
            const double u24 = 1.0 / 16777216.0;
            const double xn2 = double(xn2f);
            const double xn = sqrt(xn2);
            const double ym = double(ymf);
            // |s~ - s| <= E: tensor-core dot, FP32 key norm, score rounding
            const double E = 2.0 * eps_dot * xn * ym * 1.01 + (d + 1) * u24 * 1.02 * ym * ym +
                             2.0 * u24 * (ym * ym + 2.0 * xn * ym) * 1.01 + 1e-30;
            // lower bound on the centred squared distance of any unkept point
            const double p_lo = xn2 * (1.0 - (d + 1) * u24 * 1.02) + double(sp) - E;
            const double dist_lo =
                (p_lo > 0.0 ? sqrt(p_lo) : 0.0) - 1.02 * u24 * (xn + ym);  // centring rounding
            const double w_lo = dist_lo * (1.0 - (d + 4.0) * u24 * 1.05);  // canonical FP32 error
            cert = w_lo > double(key_w(kth));
        }
    }
    cert = __shfl_sync(0xffffffffu, cert, 0);
    if (cert) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int idx = h * 32 + lane;
            if (idx < k) {
                nbr_row[idx] = int32_t(key_lo(key[h]));
                dist_row[idx] = key_w(key[h]);
            }
        }
    }
    return cert;
}

template <int VEC, int KC, int XR>
__global__ void rerank_kernel(const float *__restrict__ X, int64_t n, int d, int k,
                              const int32_t *__restrict__ cand, const float *__restrict__ splus,
                              const float *__restrict__ skip,
                              const float *__restrict__ xnorm2, const unsigned *__restrict__ ymax_bits,
                              CertConst cc, int32_t *__restrict__ nbr, float *__restrict__ dist,
                              int32_t *__restrict__ fail_rows, int32_t *__restrict__ fail_count) {
    int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    const float sk = skip ? skip[i] : __int_as_float(0x7f800000);
    bool cert = rerank_row<VEC, KC, XR>(X, d, d, d, X + i * d, k, cand + i * (KC - 1), splus[i], sk,
                                    xnorm2[i], __uint_as_float(*ymax_bits), cc.eps_dot, lane,
                                    nbr + i * k, dist + i * k);
    if (!cert && lane == 0) fail_rows[atomicAdd(fail_count, 1)] = int32_t(i);
}

// Re-rank in the pruning's cell order: sorted row r is point i = perm[r];
// candidate rows are read from the sorted copy Xs (a row's candidates are
// mostly cell-mates, so they sit close together in memory), keyed and
// written with their original ids.
template <int VEC, int KC, int XR>
__global__ void __launch_bounds__(256, 5) rerank_sorted_kernel(const float *__restrict__ Xs, int64_t n, int d, int k,
                                     const int32_t *__restrict__ cand,
                                     const float *__restrict__ splus,
                                     const float *__restrict__ skipQ,
                                     const int32_t *__restrict__ perm,
                                     const float *__restrict__ xnorm2,
                                     const unsigned *__restrict__ ymax_bits, CertConst cc,
                                     int32_t *__restrict__ nbr, float *__restrict__ dist,
                                     int32_t *__restrict__ fail_rows,
                                     int32_t *__restrict__ fail_count) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int64_t i = perm[r];
    const bool cert = rerank_row<VEC, KC, XR>(Xs, d, d, d, Xs + r * d, k, cand + r * (KC - 1),
                                          splus[r], skipQ[r / BM], xnorm2[i],
                                          __uint_as_float(*ymax_bits), cc.eps_dot, lane,
                                          nbr + i * k, dist + i * k, perm);
    if (!cert && lane == 0) fail_rows[atomicAdd(fail_count, 1)] = int32_t(i);
}

__device__ __forceinline__ int cloud_of(const long long *__restrict__ off, int B, long long v) {
    int lo = 0, hi = B;  // off[lo] <= v < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

// Batched re-rank: one warp per compact row of a cloud that used the tensor
// tiles. Xc holds the clouds' rows back to back with row stride ld (zero
// beyond each cloud's d).
// perm (may be null): the rows are in a spatial order within each cloud and
// perm[v] is the compact id of row v; candidate ids are mapped through it
// and the results written at the original row.
template <int KC, int XR>
__global__ void rerank_batched_kernel(const float *__restrict__ Xc, int ld, int64_t N,
                                      const long long *__restrict__ voff, int B,
                                      const CloudDev *__restrict__ cl, int x3, int k,
                                      const int32_t *__restrict__ cand,
                                      const float *__restrict__ splus,
                                      const float *__restrict__ xnorm2,
                                      const unsigned *__restrict__ ymax_bits,
                                      const int32_t *__restrict__ perm,
                                      int32_t *__restrict__ nbr, float *__restrict__ dist,
                                      int32_t *__restrict__ fail_rows,
                                      int32_t *__restrict__ fail_count) {
    int64_t v = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (v >= N) return;
    const int b = cloud_of(voff, B, v);
    const CloudDev c = cl[b];
    if (!c.use_tc) return;
    const double u8 = 1.0 / 256.0;
    const double kprod = double(x3 ? 3 * c.d_pad : c.d_pad);
    const double eps = (x3 ? (3.0 * u8 * u8 + 3.0 * u8 * u8 * u8 + u8 * u8 * u8 * u8)
                           : (2.0 * u8 + u8 * u8)) +
                       kprod * (1.0 / 4194304.0) * (1.0 + 4.0 * u8);
    const int dc = (c.d + 3) & ~3;
    const int64_t pv = perm ? int64_t(perm[v]) : v;
    bool cert = rerank_row<4, KC, XR>(Xc, ld, dc, c.d, Xc + v * ld, k, cand + v * (KC - 1), splus[v],
                                  __int_as_float(0x7f800000),
                                  xnorm2[v], __uint_as_float(ymax_bits[b]), eps, lane, nbr + pv * k,
                                  dist + pv * k, perm);
    if (!cert && lane == 0) fail_rows[atomicAdd(fail_count, 1)] = int32_t(pv);
}

// Exact kNN of single rows by brute force within their cloud: one warp per
// listed row (the count lives on the device); lane l scans keys l, l+32, ...
// with canonical distances and keeps its k best (w, id) in shared memory;
// the warp then merges the 32 sorted lists. k <= 64.
constexpr int FB_WARPS = 2;  // 32 KB of static shared lists per block
__global__ void fallback_rows_kernel(const float *__restrict__ Xc, int ld,
                                     const long long *__restrict__ voff, int B,
                                     const CloudDev *__restrict__ cl, int k,
                                     const int32_t *__restrict__ rows,
                                     const int32_t *__restrict__ count,
                                     int32_t *__restrict__ nbr, float *__restrict__ dist) {
    __shared__ uint64_t lists[FB_WARPS][64][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nrows = *count;
    for (int64_t q = int64_t(blockIdx.x) * FB_WARPS + w; q < nrows;
         q += int64_t(gridDim.x) * FB_WARPS) {
        const int64_t v = rows[q];
        const int b = cloud_of(voff, B, v);
        const CloudDev c = cl[b];
        const int dc = (c.d + 3) & ~3;
        const float *xi = Xc + v * ld;
        int have = 0;
        uint64_t kth = KEY_NONE;
        for (int64_t j = c.voff + lane; j < c.voff + c.n; j += 32) {
            if (j == v) continue;
            uint64_t key = nb_key(canon_dist<4>(xi, Xc + j * ld, dc), uint32_t(j));
            if (key >= kth) continue;
            int pos = have < k ? have++ : k - 1;
            while (pos > 0 && lists[w][pos - 1][lane] > key) {
                lists[w][pos][lane] = lists[w][pos - 1][lane];
                --pos;
            }
            lists[w][pos][lane] = key;
            if (have == k) kth = lists[w][k - 1][lane];
        }
        __syncwarp();
        int head = 0;
        for (int o = 0; o < k; ++o) {
            uint64_t mine = head < have ? lists[w][head][lane] : KEY_NONE;
            uint64_t best = warp_min_u64(mine);
            if (mine == best && best != KEY_NONE) ++head;  // keys are unique (distinct ids)
            if (lane == 0) {
                nbr[v * k + o] = best == KEY_NONE ? -1 : int32_t(key_lo(best));
                dist[v * k + o] = best == KEY_NONE ? __int_as_float(0x7f800000) : key_w(best);
            }
        }
        __syncwarp();
    }
}

// Batched prep: per padded row r of the operand array, the cloud's centred
// BF16 hi (and lo) operand, its FP32 squared norm (key norms in padded rows,
// +inf on padding rows; row norms in compact rows) and the cloud's largest
// norm. mean holds the clouds' column means (B x ld).
__global__ void tc_prep_batched_kernel(const float *__restrict__ Xc, int ld, int64_t NP,
                                       const long long *__restrict__ roff,
                                       const long long *__restrict__ voff, int B,
                                       const CloudDev *__restrict__ cl, int kh_half, int x3,
                                       const float *__restrict__ mean,
                                       __nv_bfloat16 *__restrict__ H, float *__restrict__ ny,
                                       float *__restrict__ xnorm, unsigned *__restrict__ ymax_bits) {
    int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (r >= NP) return;
    const int b = cloud_of(roff, B, r);
    const CloudDev c = cl[b];
    const int64_t q = r - roff[b];
    const int kh = (x3 ? 2 : 1) * kh_half;
    __nv_bfloat16 *h = H + r * kh;
    if (q >= c.n || !c.use_tc) {
        for (int t = lane; t < kh; t += 32) h[t] = __float2bfloat16_rn(0.0f);
        if (lane == 0) ny[r] = __int_as_float(0x7f800000);
        return;
    }
    const int64_t v = voff[b] + q;
    float acc = 0.0f;
    for (int t = lane; t < kh_half; t += 32) {
        float xc = t < c.d ? __fsub_rn(Xc[v * ld + t], mean[int64_t(b) * ld + t]) : 0.0f;
        __nv_bfloat16 hi = __float2bfloat16_rn(xc);
        h[t] = hi;
        if (x3) h[kh_half + t] = __float2bfloat16_rn(__fsub_rn(xc, __bfloat162float(hi)));
        acc = fmaf(xc, xc, acc);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        ny[r] = acc;
        xnorm[v] = acc;
        // the cloud's rows all raise one word: only a row above it does
        const unsigned nb = __float_as_uint(sqrtf(acc));
        if (nb > *reinterpret_cast<volatile unsigned *>(ymax_bits + b)) atomicMax(ymax_bits + b, nb);
    }
}

// centre of every cloud (one block per cloud): the FP32 mean of up to 1024
// evenly spaced rows, eight loads in flight; the centre only has to be some
// fixed point near the cloud (every bound downstream holds for any centre)
__global__ void cloud_mean_kernel(const float *__restrict__ Xc, int ld,
                                  const CloudDev *__restrict__ cl, float *__restrict__ mean) {
    const int b = blockIdx.x;
    const CloudDev c = cl[b];
    const long long S = c.n < 1024 ? c.n : 1024;
    for (int t = threadIdx.x; t < ld; t += blockDim.x) {
        float s = 0.0f;
        if (t < c.d) {
            long long i = 0;
            for (; i + 8 <= S; i += 8) {
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = __ldg(Xc + (c.voff + (i + q) * c.n / S) * ld + t);
#pragma unroll
                for (int q = 0; q < 8; ++q) s += v[q];
            }
            for (; i < S; ++i) s += __ldg(Xc + (c.voff + i * c.n / S) * ld + t);
        }
        mean[int64_t(b) * ld + t] = t < c.d && S > 0 ? s / float(S) : 0.0f;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over row-major operand rows of `cols` elements: BF16 (boxes of 64
// elements) or, with f8, bytes (boxes of 128); 128 bytes per box row either way
bool make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int box_rows,
              bool f8 = false) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t gdim[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    cuuint64_t gstride[1] = {cuuint64_t(cols) * (f8 ? 1 : 2)};
    cuuint32_t box[2] = {cuuint32_t(f8 ? 2 * BK : BK), cuuint32_t(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void *>(base), gdim, gstride,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// keep the better of two top-1 results (the second with ids offset by k0)
__global__ void top1_merge_kernel(const int32_t *__restrict__ c2, const float *__restrict__ s2,
                                  int k0, int64_t n, int32_t *__restrict__ c,
                                  float *__restrict__ s) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (c2[i] >= 0 && s2[i] < s[i]) {
        c[i] = c2[i] + k0;
        s[i] = s2[i];
    }
}

struct TcPlan {
    int d_pad, nkb, kh, stages, kc, epi;
    int64_t nq_tiles, nk_tiles;
    size_t smem;
};

// allow8: eight epilogue warps when the candidate lists fit the merge area
// (KC <= 2 CAPB) and the larger staging area still leaves three B stages
// f8: E4M3 operand rows, 128 elements (128 bytes) per K block
TcPlan tc_plan(int64_t n, int d, int k, bool x3, bool allow8 = true, bool f8 = false) {
    TcPlan p{};
    const int kel = f8 ? 2 * BK : BK;   // elements per 128-byte K block
    p.d_pad = (d + kel - 1) / kel * kel;
    p.nkb = p.d_pad / kel;
    p.kh = (x3 ? 2 : 1) * p.d_pad;
    // keep at least ~10 candidates beyond k so that the certificate has a
    // gap to work with: k <= 21 -> 31 candidates, k <= 37 -> 47, k <= 63 -> 63
    p.kc = (k <= 21) ? 32 : (k <= 37 ? 48 : 64);
    p.nq_tiles = (n + BM - 1) / BM;
    p.nk_tiles = (n + BN - 1) / BN;
    const size_t cap = 227 * 1024;
    auto fixed_for = [&](int nh) {
        return 1024 + size_t(x3 ? 2 : 1) * p.nkb * A_BLOCK + size_t(nh) * CAPB * BM * 8 +
               2 * BM * 4 + 512;
    };
    auto stages_for = [&](size_t fixed) {
        int st = cap > fixed ? int((cap - fixed) / B_BLOCK) : 0;
        return st > 6 ? 6 : st;
    };
    const int st8 = stages_for(fixed_for(2));
    p.epi = (allow8 && p.kc <= 2 * CAPB && st8 >= 3) ? 8 : 4;
    const size_t fixed = fixed_for(p.epi / 4);
    p.stages = stages_for(fixed);
    p.smem = fixed + size_t(p.stages) * B_BLOCK;
    return p;
}

}  // namespace

bool knn_tc_supported(int64_t n, int d, int k, bool x3, bool f8) {
    if (k + 1 > 64 || n < 2) return false;
    TcPlan p = tc_plan(n, d, k, x3 && !f8, true, f8);
    return p.stages >= 2 && encode_fn() != nullptr;
}

size_t knn_tc_workspace(int64_t n, int d, int k, bool x3, int num_sms, bool prune, bool f8) {
    TcPlan p = tc_plan(n, d, k, x3 && !f8, true, f8);
    if (f8) prune = false;
    size_t b = 0;
    if (prune) {
        const int64_t K = prune_pivots_max(n), Kpad = (K + BN - 1) / BN * BN;
        b += align256(size_t(K) * 4) + align256(size_t(K) * p.kh * 2) +
             align256(size_t(Kpad + BN) * 4) * 2 + align256(size_t(n) * 4) * 2;
        b += prune_workspace(n, d, p.kh, p.kc - 1, p.nq_tiles, p.nk_tiles);
    }
    b += align256(size_t(n) * p.kh * (f8 ? 1 : 2));        // operand rows
    if (f8) b += align256(size_t(p.nk_tiles) * BN * 4);    // per-row scales
    b += align256(size_t(p.nk_tiles) * BN * 4) * 2;        // ny, components (padded)
    b += align256(size_t(n) * 4);                          // xnorm2
    b += align256(size_t(d) * 4) + 256;                    // mean, ymax
    b += align256(size_t(4096) * d * 8);                   // column partials
    b += align256(size_t(n) * (p.kc - 1) * 4);             // candidates
    b += align256(size_t(n) * 4) * 2 + 256;                // splus, fail rows, count
    b += knn_fp32_workspace(n, d, k, n, num_sms);          // fallback
    return b;
}

famst_status knn_tc(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, int k, bool x3,
                    bool vec4, int32_t *nbr, float *dist, int32_t *pinned_host,
                    int64_t *uncertified, const int32_t *colcomp, bool prune,
                    int64_t *tiles_visited, bool f8) {
    if (f8) {   // single E4M3 products, no tile pruning, no component mask
        x3 = false;
        prune = false;
        if (colcomp) return FAMST_ERR_UNSUPPORTED;
    }
    TcPlan p = tc_plan(n, d, k, x3, true, f8);
    if (p.stages < 2 || k + 1 > 64) return FAMST_ERR_UNSUPPORTED;
    // operand rows: BF16 (kh elements) or E4M3 bytes (kh bytes) with per-row scales
    __nv_bfloat16 *H = f8 ? nullptr : ar.take<__nv_bfloat16>(size_t(n) * p.kh);
    uint8_t *Q = f8 ? ar.take<uint8_t>(size_t(n) * p.kh) : nullptr;
    float *rscale = f8 ? ar.take<float>(size_t(p.nk_tiles) * BN) : nullptr;
    if (f8 && (!Q || !rscale)) return FAMST_ERR_OOM;
    float *ny = ar.take<float>(size_t(p.nk_tiles) * BN);
    float *xn2 = ar.take<float>(size_t(n));
    float *mean = ar.take<float>(size_t(d));
    unsigned *ymax = ar.take<unsigned>(1);
    const int rows_per = int((n + 4095) / 4096) > 0 ? int((n + 4095) / 4096) : 1;
    const int nb = int((n + rows_per - 1) / rows_per);
    double *part = ar.take<double>(size_t(nb) * d);
    int32_t *cand = ar.take<int32_t>(size_t(n) * (p.kc - 1));
    float *splus = ar.take<float>(size_t(n));
    int32_t *fail_rows = ar.take<int32_t>(size_t(n));
    int32_t *fail_count = ar.take<int32_t>(1);
    if ((!f8 && !H) || !ny || !xn2 || !mean || !ymax || !part || !cand || !splus || !fail_rows ||
        !fail_count)
        return FAMST_ERR_OOM;
    // prep: mean, centred BF16 operands, norms
    FAMST_LAUNCH(ex, colsum_partial_kernel, nb, 128, 0, X, n, d, rows_per, part);
    FAMST_LAUNCH(ex, colsum_final_kernel, d, 256, 0, part, nb, d, n, mean);
    if (cudaMemsetAsync(ymax, 0, 4, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(fail_count, 0, 4, ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    const int64_t npad = p.nk_tiles * BN;
    if (f8) {
        FAMST_LAUNCH(ex, tc_prep_f8_kernel, unsigned((n * 32 + 255) / 256), 256, 0, X, n, d,
                     p.d_pad, mean, Q, rscale, ny, xn2, ymax);
        if (npad > n)
            FAMST_LAUNCH(ex, fill_value_kernel, unsigned((npad - n + 255) / 256), 256, 0, rscale,
                         n, npad, 1.0f);
    } else {
        FAMST_LAUNCH(ex, tc_prep_kernel, unsigned((n * 32 + 255) / 256), 256, 0, X, n, d, p.d_pad,
                     int(x3), mean, H, ny, xn2, ymax);
    }
    if (npad > n)
        FAMST_LAUNCH(ex, fill_inf_kernel, unsigned((npad - n + 255) / 256), 256, 0, ny, n, npad);
    const bool use_prune = prune && !colcomp && prune_supported(n, d, k, vec4);
    // persistent launches: one CTA per SM takes the query tiles round-robin
    const unsigned pgrid = unsigned(std::min<int64_t>(p.nq_tiles, ex.num_sms));
    PruneOut P;
    if (use_prune) {
        // pivot cells: top-1 pivot of every point on the tensor tiles (BF16),
        // evenly spaced pivots plus two coverage passes
        const int K0 = prune_pivots(n), M = prune_extra(n), Kmax = prune_pivots_max(n);
        const int Kpadmax = (Kmax + BN - 1) / BN * BN;
        int32_t *piv = ar.take<int32_t>(size_t(Kmax));
        __nv_bfloat16 *Hp = ar.take<__nv_bfloat16>(size_t(Kmax) * p.kh);
        float *nyp = ar.take<float>(size_t(Kpadmax + BN));   // +inf beyond the pivots
        // the pass's norms copied to an aligned buffer: the tile kernel reads
        // them as float4 from tile starts, and k0 need not be a multiple of 4
        float *nya = ar.take<float>(size_t(Kpadmax + BN));
        if (!piv || !Hp || !nyp || !nya) return FAMST_ERR_OOM;
        famst_status st =
            prune_pivot_operands(ex, H, p.kh, ny, n, K0, Kpadmax + BN, piv, Hp, nyp);
        if (st != FAMST_OK) return st;
        const TcPlan p1 = tc_plan(n, d, 1, false);
        if (set_smem_attr(knn_tc_kernel<1, false>, int(p1.smem), ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        // top-1 over pivots [k0, k0 + kc) into (c_out, s_out), ids relative to k0
        auto assign = [&](int k0, int kc, int32_t *c_out, float *s_out) -> famst_status {
            CUtensorMap mA1, mB1;
            if (!make_map(&mA1, H, n, p.kh, BM) ||
                !make_map(&mB1, Hp + size_t(k0) * p.kh, kc, p.kh, BN))
                return FAMST_ERR_CUDA;
            const int nkt = (kc + BN - 1) / BN;
            if (cudaMemcpyAsync(nya, nyp + k0, size_t(nkt) * BN * 4, cudaMemcpyDeviceToDevice,
                                ex.stream) != cudaSuccess)
                return FAMST_ERR_CUDA;
            if (kc < nkt * BN)   // columns beyond the pass's pivots never win
                FAMST_LAUNCH(ex, fill_inf_kernel, 1, 256, 0, nya, int64_t(kc), int64_t(nkt) * BN);
            TcArgs a1{int(n), nkt, p.nkb, 0, p1.stages, nya, c_out, s_out,
                      ex.dstatus, nullptr, nullptr, nullptr, 1, p1.epi};
            a1.nitems = int(p.nq_tiles);   // persistent: one CTA per SM walks the query tiles
            FAMST_LAUNCH(ex, (knn_tc_kernel<1, false>), pgrid, 64 + 32 * p1.epi, p1.smem, mA1, mB1,
                         a1);
            return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
        };
        int K = K0;
        st = assign(0, K, cand, splus);
        // each coverage pass scores the points against the new pivots only
        int32_t *c2 = ar.take<int32_t>(size_t(n));
        float *s2 = ar.take<float>(size_t(n));
        if (!c2 || !s2) return FAMST_ERR_OOM;
        for (int pass = 0; pass < 2 && st == FAMST_OK; ++pass) {
            int me = 0;
            st = prune_augment(ex, ar, xn2, splus, n, H, p.kh, ny, M, K, piv, Hp, nyp, &me);
            // only the distinct new pivots are scored (the repeats add no cell)
            if (st == FAMST_OK && me > 0) {
                st = assign(K, me, c2, s2);
                if (st == FAMST_OK)
                    FAMST_LAUNCH(ex, top1_merge_kernel, unsigned((n + 255) / 256), 256, 0, c2, s2,
                                 K, n, cand, splus);
            }
            K += M;
        }
        if (st != FAMST_OK) return st;
        st = prune_partition(ex, ar, X, d, n, k, H, p.kh, ny, p.nkb, K, piv, cand, 1,
                             pinned_host + 2, &P);
        if (st != FAMST_OK) return st;
    }
    // candidates of the tensor pass: directly in cand / splus, or (pruned)
    // in sorted order first
    int32_t *cand_t = cand;
    float *splus_t = splus;
    int32_t *side_j = nullptr;   // candidates of the parts of split lists
    float *side_s = nullptr, *side_sp = nullptr;
    if (use_prune) {
        cand_t = ar.take<int32_t>(size_t(n) * (p.kc - 1));
        splus_t = ar.take<float>(size_t(n));
        side_j = ar.take<int32_t>(size_t(PRUNE_SPLIT_SLOTS) * BM * (p.kc - 1));
        side_s = ar.take<float>(size_t(PRUNE_SPLIT_SLOTS) * BM * (p.kc - 1));
        side_sp = ar.take<float>(size_t(PRUNE_SPLIT_SLOTS) * BM);
        if (!cand_t || !splus_t || !side_j || !side_s || !side_sp) return FAMST_ERR_OOM;
    }
    const void *Hop = f8 ? static_cast<const void *>(Q)
                         : static_cast<const void *>(use_prune ? P.Hs : H);
    CUtensorMap mA, mB;
    if (!make_map(&mA, Hop, n, p.kh, BM, f8) || !make_map(&mB, Hop, n, p.kh, BN, f8))
        return FAMST_ERR_CUDA;
    int32_t *cpad = nullptr;   // components over the padded rows (-1 beyond n)
    if (colcomp) {
        cpad = ar.take<int32_t>(size_t(npad));
        if (cudaMemsetAsync(cpad, 0xff, size_t(npad) * 4, ex.stream) != cudaSuccess ||
            cudaMemcpyAsync(cpad, colcomp, size_t(n) * 4, cudaMemcpyDeviceToDevice, ex.stream) !=
                cudaSuccess)
            return FAMST_ERR_CUDA;
    }
    // certificate constants (also the pruned lists' start thresholds)
    const double u8 = 1.0 / 256.0;
    const double kprod = double(x3 ? 3 * p.d_pad : p.d_pad);
    CertConst cc;
    cc.eps_dot = (x3 ? (3.0 * u8 * u8 + 3.0 * u8 * u8 * u8 + u8 * u8 * u8 * u8)
                     : (2.0 * u8 + u8 * u8)) +
                 kprod * std::ldexp(1.0, -22) * (1.0 + 4.0 * u8);
    if (f8) {
        // E4M3 with the row's scale: a normal element is within u = 2^-4 of
        // x'_t (relative); an element below the normal range within 2^-10 s,
        // and s <= 2 max|x'| / 448, so over the row those add at most
        // sqrt(d) 2^-10 (2 / 448) ||x'|| per side. Products of E4M3 values
        // are exact in FP32; the accumulation term is as for BF16.
        // With |x^_t - x'_t| <= u|x'_t| + c ||x'|| (c = 2^-10 2/448) on both
        // sides, |x^.y^ - x'.y'| <= ((2u + u^2) + 2 sqrt(d)(1 + u) c + d c^2)
        // ||x'|| ||y'||.
        const double u4 = 1.0 / 16.0, c8 = 2.0 / 448.0 / 1024.0, dp = double(p.d_pad);
        cc.eps_dot = 2.0 * u4 + u4 * u4 + 2.0 * std::sqrt(dp) * (1.0 + u4) * c8 + dp * c8 * c8 +
                     kprod * std::ldexp(1.0, -22) * (1.0 + 4.0 * u4);
    }
    cc.d_plus = double(d) + 4.0;
    if (use_prune)
        FAMST_LAUNCH(ex, thr0_kernel, unsigned((n + 255) / 256), 256, 0, P.tau_row, P.nys, n, d,
                     ymax, cc.eps_dot);
    TcArgs a{int(n), int(p.nk_tiles), p.nkb, int(x3), p.stages, use_prune ? P.nys : ny, cand_t,
             splus_t, ex.dstatus, use_prune ? P.tab : nullptr, cpad,
             use_prune ? P.klist : nullptr, 0, p.epi, rscale, use_prune ? P.tau_row : nullptr};
    // one CTA per work item: the pruned tiles' key lists differ in length,
    // and a static round-robin over persistent CTAs measured slower here.
    // Pruned lists come as work items, long ones split into parts; the grid
    // covers the most items the table can hold and the CTAs beyond its
    // count leave at once.
    unsigned tgrid = unsigned(p.nq_tiles);
    if (use_prune) {
        a.nitems_dev = P.nitems;
        a.side_j = side_j;
        a.side_s = side_s;
        a.side_splus = side_sp;
        tgrid = unsigned(p.nq_tiles + PRUNE_SPLIT_SLOTS);
    }
#define TC_LAUNCH(KCV, M)                                                                        \
    do {                                                                                         \
        if (set_smem_attr(knn_tc_kernel<KCV, M>, int(p.smem), ex.stream) != cudaSuccess)         \
            return FAMST_ERR_CUDA;                                                               \
        FAMST_LAUNCH(ex, (knn_tc_kernel<KCV, M>), tgrid, 64 + 32 * p.epi, p.smem, mA, mB, a);   \
    } while (0)
#define TC_LAUNCH_F8(KCV)                                                                           \
    do {                                                                                            \
        if (set_smem_attr(knn_tc_kernel<KCV, false, true>, int(p.smem), ex.stream) != cudaSuccess)  \
            return FAMST_ERR_CUDA;                                                                  \
        FAMST_LAUNCH(ex, (knn_tc_kernel<KCV, false, true>), tgrid, 64 + 32 * p.epi,                \
                     p.smem, mA, mB, a);                                                            \
    } while (0)
    timer_mark(ex, TIMER_TILES, false);
    if (f8) {
        if (p.kc == 32) TC_LAUNCH_F8(32);
        else if (p.kc == 48) TC_LAUNCH_F8(48);
        else TC_LAUNCH_F8(64);
    } else if (cpad) {
        if (p.kc == 32) TC_LAUNCH(32, true);
        else if (p.kc == 48) TC_LAUNCH(48, true);
        else TC_LAUNCH(64, true);
    } else {
        if (p.kc == 32) TC_LAUNCH(32, false);
        else if (p.kc == 48) TC_LAUNCH(48, false);
        else TC_LAUNCH(64, false);
    }
    if (use_prune) {   // rows of split lists: merge their parts
#define SPLIT_MERGE(KCV)                                                                        \
    FAMST_LAUNCH(ex, split_merge_kernel<KCV>, unsigned(PRUNE_SPLIT_TILES), BM, 0, P.splitq,     \
                 P.nsplit, side_j, side_s, side_sp, n, cand_t, splus_t)
        if (p.kc == 32) SPLIT_MERGE(32);
        else if (p.kc == 48) SPLIT_MERGE(48);
        else SPLIT_MERGE(64);
#undef SPLIT_MERGE
    }
    timer_mark(ex, TIMER_TILES, true);
#undef TC_LAUNCH
#undef TC_LAUNCH_F8
    if (cudaPeekAtLastError() != cudaSuccess) return FAMST_ERR_CUDA;
    const unsigned rgrid = unsigned((n * 32 + 255) / 256);
#define RERANK3(V, KCV, XRV)                                                                     \
    do {                                                                                         \
        if (use_prune)                                                                           \
            FAMST_LAUNCH(ex, (rerank_sorted_kernel<V, KCV, XRV>), rgrid, 256, 0, P.Xs, n, d, k,  \
                         cand_t, splus_t, P.skipQ, P.perm, xn2, ymax, cc, nbr, dist, fail_rows,  \
                         fail_count);                                                            \
        else                                                                                     \
            FAMST_LAUNCH(ex, (rerank_kernel<V, KCV, XRV>), rgrid, 256, 0, X, n, d, k, cand,      \
                         splus, nullptr, xn2, ymax, cc, nbr, dist, fail_rows, fail_count);       \
    } while (0)
#define RERANK(V, KCV)                                                                           \
    do {                                                                                         \
        if (d <= 128) RERANK3(V, KCV, 4);                                                        \
        else if (d <= 256) RERANK3(V, KCV, 8);                                                   \
        else if (d <= 512) RERANK3(V, KCV, 16);                                                  \
        else RERANK3(V, KCV, 0);                                                                 \
    } while (0)
    timer_mark(ex, TIMER_RERANK, false);
    if (p.kc == 32) {
        RERANK(1, 32);
    } else if (p.kc == 48) {
        RERANK(1, 48);
    } else {
        RERANK(1, 64);
    }
    timer_mark(ex, TIMER_RERANK, true);
#undef RERANK
#undef RERANK3
    if (cudaMemcpyAsync(pinned_host, fail_count, 4, cudaMemcpyDeviceToHost, ex.stream) != cudaSuccess ||
        (use_prune && cudaMemcpyAsync(pinned_host + 1, P.visited, 4, cudaMemcpyDeviceToHost,
                                      ex.stream) != cudaSuccess) ||
        cudaStreamSynchronize(ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    const int32_t nfail = *pinned_host;
    *uncertified = nfail;
    if (tiles_visited) *tiles_visited = use_prune ? int64_t(pinned_host[1]) : p.nq_tiles * p.nk_tiles;
    if (nfail > 0) {
        famst_status st = knn_fp32(ex, ar, X, n, d, k, fail_rows, 0, nfail, nbr, dist, colcomp);
        if (st != FAMST_OK) return st;
    }
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst

namespace famst {

// Shared-memory plan of the batched tensor path for operand width D (the
// largest cloud's K extent).
bool knn_tc_batched_plan(int D, int k, bool x3, int epi_req, int *stages, size_t *smem, int *kc,
                         int *epi) {
    if (k + 1 > 64) return false;
    TcPlan p = tc_plan(int64_t(1) << 20, D, k, x3, epi_req == 8);
    if (p.stages < 2 || encode_fn() == nullptr) return false;
    *stages = p.stages;
    *smem = p.smem;
    *kc = p.kc;
    *epi = p.epi;
    return true;
}

// The batched tile pass alone (one persistent launch over the (cloud, query
// tile) items): the autotuner times it per shape on the batch's own data.
famst_status knn_tc_batched_tiles(const Exec &ex, int D, bool x3, int stages, size_t smem, int kc,
                                  int epi, const TcTile *tiles, int64_t nctas, const float *ny,
                                  int32_t *cand, float *splus, const CUtensorMap *mA,
                                  const CUtensorMap *mB, bool spiral) {
    if (nctas <= 0) return FAMST_OK;
    const int nkb = D / BK;
    TcArgs a{0, 0, nkb, int(x3), stages, ny, cand, splus, ex.dstatus, tiles, nullptr, nullptr, 0,
             epi};
    // persistent: one CTA per SM walks the (cloud, query tile) items round-robin
    a.nitems = int(nctas);
    a.spiral = spiral ? 1 : 0;
    const unsigned bgrid = unsigned(std::min<int64_t>(nctas, ex.num_sms));
#define TCB_LAUNCH(KCV)                                                                          \
    do {                                                                                         \
        if (set_smem_attr(knn_tc_kernel<KCV, false>, int(smem), ex.stream) != cudaSuccess)      \
            return FAMST_ERR_CUDA;                                                               \
        FAMST_LAUNCH(ex, (knn_tc_kernel<KCV, false>), bgrid, 64 + 32 * epi, smem, *mA, *mB, a);  \
    } while (0)
    if (kc == 32) TCB_LAUNCH(32);
    else if (kc == 48) TCB_LAUNCH(48);
    else TCB_LAUNCH(64);
#undef TCB_LAUNCH
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

// Everything of the batched tensor path that runs on the device; buffers
// come from the caller's plan, so nothing here allocates or synchronises.
famst_status knn_tc_batched(const Exec &ex, const float *Xc, int D, int64_t N, int64_t NP,
                            const long long *voff, const long long *roff, int B,
                            const CloudDev *cl, const TcTile *tiles, int64_t nctas, int k,
                            bool x3, int stages, size_t smem, int kc, int epi, __nv_bfloat16 *H,
                            float *ny, float *xn2, float *mean, unsigned *ymax, int32_t *cand,
                            float *splus, int32_t *fail_rows, int32_t *fail_count, int32_t *nbr,
                            float *dist, const CUtensorMap *mA, const CUtensorMap *mB,
                            const float *Xorig, const int32_t *perm) {
    FAMST_LAUNCH(ex, cloud_mean_kernel, B, 128, 0, Xc, D, cl, mean);
    if (cudaMemsetAsync(ymax, 0, size_t(B) * 4, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(fail_count, 0, 4, ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, tc_prep_batched_kernel, unsigned((NP * 32 + 255) / 256), 256, 0, Xc, D, NP,
                 roff, voff, B, cl, D, int(x3), mean, H, ny, xn2, ymax);
    famst_status st = knn_tc_batched_tiles(ex, D, x3, stages, smem, kc, epi, tiles, nctas, ny, cand,
                                           splus, mA, mB, perm != nullptr);
    if (st != FAMST_OK) return st;
    const unsigned rgrid = unsigned((N * 32 + 255) / 256);
    // one candidate at a time per warp over coalesced row reads when the
    // padded rows fit the register slices (D <= 512), else one per lane
#define RRB(KCV, XRV)                                                                            \
    FAMST_LAUNCH(ex, (rerank_batched_kernel<KCV, XRV>), rgrid, 256, 0, Xc, D, N, voff, B, cl,    \
                 int(x3), k, cand, splus, xn2, ymax, perm, nbr, dist, fail_rows, fail_count)
#define RRB_KC(KCV)                                                                              \
    do {                                                                                         \
        if (D <= 128) RRB(KCV, 4);                                                               \
        else if (D <= 256) RRB(KCV, 8);                                                          \
        else if (D <= 512) RRB(KCV, 16);                                                         \
        else RRB(KCV, 0);                                                                        \
    } while (0)
    if (kc == 32) RRB_KC(32);
    else if (kc == 48) RRB_KC(48);
    else RRB_KC(64);
#undef RRB_KC
#undef RRB
    // rows no certificate covers: exact within their cloud, original order and ids
    FAMST_LAUNCH(ex, fallback_rows_kernel, unsigned(ex.num_sms) * 16, FB_WARPS * 32, 0,
                 Xorig ? Xorig : Xc, D, voff, B, cl, k, fail_rows, fail_count, nbr, dist);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

famst_status fallback_rows_batched(const Exec &ex, const float *Xc, int ld, const long long *voff,
                                   int B, const CloudDev *cl, int k, const int32_t *rows,
                                   const int32_t *count, int32_t *nbr, float *dist) {
    FAMST_LAUNCH(ex, fallback_rows_kernel, unsigned(ex.num_sms) * 16, FB_WARPS * 32, 0, Xc, ld,
                 voff, B, cl, k, rows, count, nbr, dist);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

// Tensor maps over the padded operand rows (queries 128-row boxes, keys
// 256-row boxes); made on the host before any capture.
bool knn_tc_batched_maps(const void *H, int64_t NP, int D, bool x3, CUtensorMap *mA,
                         CUtensorMap *mB) {
    const int64_t kh = (x3 ? 2 : 1) * int64_t(D);
    return make_map(mA, H, NP, kh, BM) && make_map(mB, H, NP, kh, BN);
}

}  // namespace famst
