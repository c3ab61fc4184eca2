// Algorithm 4 inside a build: the refinement scans with candidate rows staged
// in shared memory by the copy engine.
//
// A scan of Algorithm 4 looks for the u' in G[u] minimising w(u', v) (and
// then the v' in G[v] against the new u*). Its cost is the gather of the
// candidates' rows. Here:
//  * G[c] is stored once per vertex as one deduplicated list (the kNN list
//    of c followed by the reverse entries that are not already in it), each
//    entry with the id, the error bound eb and the norm ||h||^2 of the
//    candidate's centred BF16 row h: the scan reads 12 bytes per candidate
//    in list order instead of looking them up;
//  * one warp scans 32 candidates per round: every lane issues ONE bulk copy
//    (cp.async.bulk, the copy engine) of its candidate's BF16 row into the
//    warp's shared-memory buffer, counted on the warp's mbarrier; the lanes
//    then wait once per round, so all 32 row fetches are in flight together
//    and cost no registers;
//  * the 32 dot products h_c . h_fixed are two mma.sync m16n8k16 tiles per
//    16-element k step (A = 16 candidate rows read with ldmatrix, B column
//    0 = the fixed row, held in registers for the whole scan);
//  * bounds in the distance domain rule candidates out as in the register
//    filter, and the survivors are decided on canonical FP32 distances (the
//    fixed row's slices stay in registers; up to four survivors' rows are
//    fetched together).
// The result of every scan is the argmin under (w, 1 + id) with the
// incumbent keyed (w0, 0), so it equals the oracle's ascending scan with
// strict "<"; edges are iterated to their fixed points as in refine_kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "famst_internal.cuh"
#include "mbarrier.cuh"

namespace famst {
namespace {

// ------------------------------------------------------------- G lists

// |G[c]| = k + (reverse entries r of c with r not in nbr[c]); one warp per c
__global__ void glist_count_kernel(const int32_t *__restrict__ nbr, int64_t n, int k,
                                   const int32_t *__restrict__ rev_off,
                                   const int32_t *__restrict__ rev_src, int32_t *__restrict__ cnt) {
    const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    const int r0 = rev_off[c], r1 = rev_off[c + 1];
    const int32_t *nb = nbr + c * k;
    int kept = 0;
    for (int base = r0; base < r1; base += 32) {
        const int idx = base + lane;
        bool keep = false;
        if (idx < r1) {
            const int32_t r = rev_src[idx];
            keep = true;
            for (int j = 0; j < k; ++j) keep &= (__ldg(nb + j) != r);
        }
        kept += __popc(__ballot_sync(0xffffffffu, keep));
    }
    if (lane == 0) cnt[c] = k + kept;
}

__global__ void glist_fill_kernel(const int32_t *__restrict__ nbr, int64_t n, int k,
                                  const int32_t *__restrict__ rev_off,
                                  const int32_t *__restrict__ rev_src,
                                  const int32_t *__restrict__ goff, const float *__restrict__ eb,
                                  const float *__restrict__ n2, int32_t *__restrict__ gid,
                                  float2 *__restrict__ gen) {
    const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    const int64_t o = goff[c];
    const int32_t *nb = nbr + c * k;
    for (int j = lane; j < k; j += 32) {
        const int32_t y = nb[j];
        gid[o + j] = y;
        gen[o + j] = make_float2(eb[y], n2[y]);
    }
    const int r0 = rev_off[c], r1 = rev_off[c + 1];
    int64_t pos = o + k;
    for (int base = r0; base < r1; base += 32) {
        const int idx = base + lane;
        bool keep = false;
        int32_t r = -1;
        if (idx < r1) {
            r = rev_src[idx];
            keep = true;
            for (int j = 0; j < k; ++j) keep &= (__ldg(nb + j) != r);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int64_t s = pos + __popc(m & ((1u << lane) - 1u));
            gid[s] = r;
            gen[s] = make_float2(eb[r], n2[r]);
        }
        pos += __popc(m);
    }
}

// ------------------------------------------------------------ the scan

// rows of the staging buffer: ld BF16 values + 16 bytes of padding, so the
// 8 rows an ldmatrix phase reads fall in 8 different 16-byte bank groups
template <int NKS>
struct Stage {
    static constexpr int LD = NKS * 16;         // row length (elements)
    static constexpr int RS = LD * 2 + 16;      // row stride in shared memory (bytes)
    static constexpr int WARP_BYTES = 32 * RS;  // one round of 32 candidates
    static constexpr int WARPS = NKS >= 16 ? 4 : 8;
    static constexpr int SMEM = 128 + WARPS * WARP_BYTES;
};

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &a0, uint32_t &a1, uint32_t &a2,
                                        uint32_t &a3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                 : "r"(addr)
                 : "memory");
}

__device__ __forceinline__ uint32_t ldg_u32(const __nv_bfloat16 *p) {
    return __ldg(reinterpret_cast<const unsigned int *>(p));
}

struct ScanOut {
    uint64_t best;
    bool dead;   // a bounded wait expired (the kernel stops)
};

// argmin over G[c] of (w(c', fixed), 1 + c') with the incumbent (w0, 0).
// XR > 0: d <= 32 XR, the fixed row's FP32 slices stay in registers.
template <int NKS, int XR>
__device__ __forceinline__ ScanOut scan_bulk(
    const float *__restrict__ X, int d, int c, int fixed, float w0, const GLists &g,
    const __nv_bfloat16 *__restrict__ H, const float *__restrict__ heb,
    const float *__restrict__ hn2, char *buf, uint64_t *bar, uint32_t &phase, int lane, float aerr,
    float eps, unsigned &evals, unsigned &canon, int *dstatus) {
    using S = Stage<NKS>;
    const __nv_bfloat16 *hf = H + int64_t(fixed) * S::LD;
    // B fragments of m16n8k16: column 0 holds the fixed row (lanes 0-3 carry
    // k pairs (2t, 2t+1) and (8+2t, 9+2t) of each k step), columns 1-7 zero
    uint32_t b0[NKS], b1[NKS];
#pragma unroll
    for (int ks = 0; ks < NKS; ++ks) {
        b0[ks] = lane < 4 ? ldg_u32(hf + 16 * ks + 2 * lane) : 0u;
        b1[ks] = lane < 4 ? ldg_u32(hf + 16 * ks + 8 + 2 * lane) : 0u;
    }
    const float ebx = __ldg(heb + fixed), nx = __ldg(hn2 + fixed);
    const float *xf = X + int64_t(fixed) * d;
    float xr[XR > 0 ? XR : 1];
#pragma unroll
    for (int q = 0; q < XR; ++q) {
        const int t = lane + 32 * q;
        xr[q] = t < d ? __ldg(xf + t) : 0.0f;
    }
    uint64_t best = uint64_t(__float_as_uint(w0)) << 32;
    const int base = g.off[c], deg = g.off[c + 1] - base;
    const float inf = __int_as_float(0x7f800000);
    const uint32_t sbuf = smem_u32(buf);
    // ldmatrix row of this lane: matrix lane/8 = (rows 8 (mi & 1).., k half mi >> 1)
    const int mi = lane >> 3, rr = lane & 7;
    const uint32_t arow = sbuf + uint32_t(((mi & 1) * 8 + rr) * S::RS + (mi >> 1) * 16);
    for (int r0 = 0; r0 < deg; r0 += 32) {
        const int idx = r0 + lane;
        const bool valid = idx < deg;
        int cand = -1;
        float2 en = make_float2(0.0f, 0.0f);
        if (valid) {
            cand = __ldg(g.id + base + idx);
            en = __ldg(g.en + base + idx);
        }
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) {
            mbar_expect_tx(bar, uint32_t(__popc(vm)) * uint32_t(S::LD * 2));
            evals += unsigned(__popc(vm));
        }
        __syncwarp();
        if (valid) bulk_load(buf + lane * S::RS, H + int64_t(cand) * S::LD, S::LD * 2, bar);
        if (!__all_sync(0xffffffffu, mbar_drain(bar, phase))) {
            // the copies did not land in time: flag it, give them one more
            // bounded wait, and stop (the decision is the whole warp's)
            if (lane == 0) set_status(dstatus, STATUS_LOOP_LIMIT);
            mbar_drain(bar, phase);
            return ScanOut{best, true};
        }
        phase ^= 1u;
        // dot products: tile T holds candidates 16 T .. 16 T + 15
        float acc[2][4];
#pragma unroll
        for (int T = 0; T < 2; ++T) {
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[T][e] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < NKS; ++ks) {
                uint32_t a0, a1, a2, a3;
                ldsm_x4(arow + uint32_t(T * 16 * S::RS + ks * 32), a0, a1, a2, a3);
                mma_bf16_16816(acc[T], a0, a1, a2, a3, b0[ks], b1[ks]);
            }
        }
        __syncwarp();   // every lane's ldmatrix is done before the next round's copies
        // D column 0: lane 4 g holds rows g (acc[.][0]) and g + 8 (acc[.][2]);
        // candidate j = 16 T + r comes from lane 4 (r mod 8)
        const int src = 4 * (lane & 7);
        const float v00 = __shfl_sync(0xffffffffu, acc[0][0], src);
        const float v02 = __shfl_sync(0xffffffffu, acc[0][2], src);
        const float v10 = __shfl_sync(0xffffffffu, acc[1][0], src);
        const float v12 = __shfl_sync(0xffffffffu, acc[1][2], src);
        const float dt = lane < 16 ? ((lane & 8) ? v02 : v00) : ((lane & 8) ? v12 : v10);
        // bounds on the canonical distance (see scan_side_filtered)
        float lo = inf, hi = inf;
        if (valid) {
            const float nn = __fadd_rn(nx, en.y);
            const float pt = __fmaf_rn(-2.0f, dt, nn);
            const float A = __fmaf_ru(nn, aerr, 1e-35f);
            const float slo = __fsqrt_rd(fmaxf(__fsub_rd(pt, A), 0.0f));
            const float shi = __fsqrt_ru(__fadd_ru(pt, A));
            const float E = __fadd_ru(ebx, en.x);
            lo = fmaxf(__fmul_rd(__fsub_rd(slo, E), 1.0f - eps), 0.0f);
            hi = __fmul_ru(__fadd_ru(shi, E), 1.0f + eps);
        }
        float mh = hi;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) mh = fminf(mh, __shfl_xor_sync(0xffffffffu, mh, o));
        const float bound = __fmul_ru(fminf(mh, key_w(best)), 1.0f + 0x1p-22f);
        unsigned sv = __ballot_sync(0xffffffffu, valid && lo <= bound);
        if (lane == 0) canon += unsigned(__popc(sv));
        // survivors: canonical distances by the whole warp, up to four rows
        // fetched together
        while (sv) {
            if constexpr (XR > 0) {
                int cs[4];
                float yv[4][XR];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cs[j] = -1;
                    if (sv) {
                        const int sl = __ffs(sv) - 1;
                        sv &= sv - 1;
                        cs[j] = __shfl_sync(0xffffffffu, cand, sl);
                    }
                    const float *yr = X + int64_t(cs[j] >= 0 ? cs[j] : fixed) * d;
#pragma unroll
                    for (int q = 0; q < XR; ++q) {
                        const int t = lane + 32 * q;
                        yv[j][q] = (cs[j] >= 0 && t < d) ? __ldg(yr + t) : 0.0f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (cs[j] < 0) continue;
                    float p = 0.0f;
#pragma unroll
                    for (int q = 0; q < XR; ++q) {
                        const float dl = __fsub_rn(yv[j][q], xr[q]);
                        p = __fmaf_rn(dl, dl, p);
                    }
#pragma unroll
                    for (int o = 16; o >= 1; o >>= 1)
                        p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
                    const float w = __fsqrt_rn(p);
                    const uint64_t key =
                        (uint64_t(__float_as_uint(w)) << 32) | uint32_t(cs[j] + 1);
                    best = key < best ? key : best;
                }
            } else {
                const int sl = __ffs(sv) - 1;
                sv &= sv - 1;
                const int c2 = __shfl_sync(0xffffffffu, cand, sl);
                const float w = __fsqrt_rn(canon_p_warp(X + int64_t(c2) * d, xf, d, lane));
                const uint64_t key = (uint64_t(__float_as_uint(w)) << 32) | uint32_t(c2 + 1);
                best = key < best ? key : best;
            }
        }
    }
    return ScanOut{best, false};
}

// Edges handed out one at a time (in component-pair tile order, so the rows
// in flight stay in L2), each iterated to its own fixed point; the v-scan
// of a sweep that repeats the previous sweep's inputs is reused.
template <int NKS, int XR, int MINB>
__global__ void __launch_bounds__(Stage<NKS>::WARPS * 32, MINB)
    refine_bulk_kernel(const float *__restrict__ X, int d, GLists g,
                       const __nv_bfloat16 *__restrict__ H, const float *__restrict__ heb,
                       const float *__restrict__ hn2, int32_t *__restrict__ eu,
                       int32_t *__restrict__ ev, float *__restrict__ ew,
                       const int32_t *__restrict__ order, int64_t m, int max_iters,
                       int32_t *__restrict__ change_hist,
                       unsigned long long *__restrict__ next_item, int *dstatus,
                       unsigned long long *__restrict__ evals_out, float aerr, float eps) {
    using S = Stage<NKS>;
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem) + warp;
    char *buf = smem + 128 + warp * S::WARP_BYTES;
    if (lane == 0) mbar_init(bar, 1);
    mbar_init_fence();
    __syncwarp();
    uint32_t phase = 0;
    unsigned long long evals_total = 0, canon_total = 0;
    bool dead = false;
    while (!dead) {
        unsigned long long w0 = 0;
        if (lane == 0) w0 = atomicAdd(next_item, 1ull);
        const int64_t w = int64_t(__shfl_sync(0xffffffffu, w0, 0));
        if (w >= m) break;
        const int64_t e = order ? int64_t(order[w]) : w;
        int u = eu[e], v = ev[e];
        float wt = ew[e];
        int changes = 0;
        unsigned evals = 0, canon = 0;
        int mv_v = -1, mv_u = -1;
        uint64_t mv_b = 0;
        for (; changes < max_iters; ++changes) {
            // u-loop: u' in G[u] against v
            ScanOut su = scan_bulk<NKS, XR>(X, d, u, v, wt, g, H, heb, hn2, buf, bar, phase, lane,
                                            aerr, eps, evals, canon, dstatus);
            if (su.dead) { dead = true; break; }
            const int us = key_lo(su.best) ? int(key_lo(su.best)) - 1 : u;
            float ws = key_w(su.best);
            // v-loop: v' in G[v] against the new u*
            uint64_t bv;
            if (v == mv_v && us == mv_u) {
                bv = mv_b;
            } else {
                ScanOut sw = scan_bulk<NKS, XR>(X, d, v, us, ws, g, H, heb, hn2, buf, bar, phase,
                                                lane, aerr, eps, evals, canon, dstatus);
                if (sw.dead) { dead = true; break; }
                bv = sw.best;
            }
            mv_v = v;
            mv_u = us;
            mv_b = bv;
            const int vs = key_lo(bv) ? int(key_lo(bv)) - 1 : v;
            ws = key_w(bv);
            if (us == u && vs == v) break;
            u = us;
            v = vs;
            wt = ws;
        }
        if (dead) break;
        if (lane == 0) {
            eu[e] = u;
            ev[e] = v;
            ew[e] = wt;
            atomicAdd(&change_hist[changes], 1);
            if (changes == max_iters) set_status(dstatus, STATUS_REFINE_CAP);
        }
        evals_total += evals;
        canon_total += canon;
    }
    if (evals_out && lane == 0) {   // [0] candidate distances, [1] canonical evaluations
        atomicAdd(evals_out, evals_total);
        atomicAdd(evals_out + 1, canon_total);
    }
}

}  // namespace

size_t glists_workspace(int64_t n, int k) {
    return 2 * align256(size_t(n + 1) * 4) + scan_workspace(n) + align256(size_t(n) * k * 2 * 4) +
           align256(size_t(n) * k * 2 * 8);
}

famst_status refine_glists(const Exec &ex, Arena &ar, const int32_t *nbr, int64_t n, int k,
                           const int32_t *rev_off, const int32_t *rev_src, HalfRows *hr) {
    if (!hr->h) return FAMST_OK;
    int32_t *cnt = ar.take<int32_t>(size_t(n + 1));
    int32_t *goff = ar.take<int32_t>(size_t(n + 1));
    int32_t *gid = ar.take<int32_t>(size_t(n) * k * 2);
    float2 *gen = ar.take<float2>(size_t(n) * k * 2);
    if (!cnt || !goff || !gid || !gen) return FAMST_ERR_OOM;
    const unsigned gr = unsigned((n * 32 + 255) / 256);
    FAMST_LAUNCH(ex, glist_count_kernel, gr, 256, 0, nbr, n, k, rev_off, rev_src, cnt);
    famst_status st = exclusive_scan_i32(ex, ar, cnt, goff, n, goff + n);
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, glist_fill_kernel, gr, 256, 0, nbr, n, k, rev_off, rev_src, goff, hr->eb,
                 hr->n2, gid, gen);
    hr->g = GLists{goff, gid, gen};
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

bool refine_bulk_supported(const HalfRows &hr) {
    return hr.h && hr.g.id && (hr.ld == 64 || hr.ld == 128 || hr.ld == 256);
}

famst_status launch_refine_bulk(const Exec &ex, const float *X, int d, const HalfRows &hr,
                                int32_t *eu, int32_t *ev, float *ew, const int32_t *order,
                                int64_t m, int max_iters, int32_t *change_hist,
                                unsigned long long *next_item, unsigned long long *evals) {
    // canonical distance vs the exact one, generously: (d + 16) u
    const float eps = float((d + 16) * std::ldexp(1.0, -24) * 1.1);
    const float aerr = float(hr.ld * std::ldexp(1.0, -19) + std::ldexp(1.0, -20));
    const void *fn;
    int threads, smem;
#define RB_PICK(NK, XRV, MB)                                                  \
    do {                                                                      \
        fn = (const void *)refine_bulk_kernel<NK, XRV, MB>;                   \
        threads = Stage<NK>::WARPS * 32;                                      \
        smem = Stage<NK>::SMEM;                                               \
        if (set_smem_attr(refine_bulk_kernel<NK, XRV, MB>, smem, ex.stream) != \
            cudaSuccess)                                                      \
            return FAMST_ERR_CUDA;                                            \
    } while (0)
    if (hr.ld == 64) RB_PICK(4, 2, 4);
    else if (hr.ld == 128) RB_PICK(8, 4, 3);
    else RB_PICK(16, 0, 2);
#undef RB_PICK
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t warps = int64_t(threads / 32);
    int64_t want = (m + warps - 1) / warps;
    int64_t cap = int64_t(ex.num_sms) * per_sm;
    unsigned grid = unsigned(want < cap ? want : cap);
    if (grid == 0) grid = 1;
    GLists g = hr.g;
#define RB_LAUNCH(NK, XRV, MB)                                                                 \
    FAMST_LAUNCH(ex, (refine_bulk_kernel<NK, XRV, MB>), grid, threads, smem, X, d, g, hr.h,  \
                 hr.eb, hr.n2, eu, ev, ew, order, m, max_iters, change_hist, next_item,      \
                 ex.dstatus, evals, aerr, eps)
    timer_mark(ex, TIMER_REFINE, false);
    if (hr.ld == 64) RB_LAUNCH(4, 2, 4);
    else if (hr.ld == 128) RB_LAUNCH(8, 4, 3);
    else RB_LAUNCH(16, 0, 2);
    timer_mark(ex, TIMER_REFINE, true);
#undef RB_LAUNCH
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst
