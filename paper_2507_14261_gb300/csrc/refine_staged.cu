// Algorithm 4 inside a build, with candidate rows staged in shared memory.
//
// A scan of Algorithm 4 looks for the u' in G[u] minimising w(u', v) (and
// then the v' in G[v] against the new u*). Its cost is the gather of the
// candidates' rows, so both kernels here are built around moving as few of
// those bytes as possible:
//  * G[c] is stored once per vertex as one deduplicated list (the kNN list
//    of c followed by the reverse entries that are not already in it), each
//    entry with the id, the error bound eb and the norm ||h||^2 of the
//    candidate's centred BF16 row h;
//  * a warp stages 32 candidate rows per round in shared memory (cp.async,
//    16-byte pieces, each instruction copying whole row pieces) and takes
//    the dot products on the tensor cores: mma.sync m16n8k16 with A = 16
//    candidate rows (ldmatrix) and B = up to eight fixed rows, one per
//    column;
//  * bounds in the distance domain rule candidates out (BF16 rounding of
//    both rows, accumulation error, canonical-sum error), and the survivors
//    are decided on canonical FP32 distances.
// Every scan's result is the argmin under (w, 1 + id) with the incumbent
// keyed (w0, 0), which equals the oracle's ascending scan with strict "<".
//
// Schedule. Edges do not interact (Algorithm 4), so a build runs the first
// sweeps sweep-synchronously, as the paper states them: all u-scans of the
// sweep, then all v-scans. The scans of a phase are grouped by the vertex c
// they scan: one warp loads G[c]'s rows once and scores them against the
// fixed points of every scan of c, eight per mma (on the 1M-point sphere
// mixture about five scans share a vertex in the early sweeps). Vertices are
// visited in component order, so the rows in flight belong to a few
// clusters and stay in L2. Once few edges remain active, the per-edge kernel
// iterates each of them to its fixed point in one launch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "famst_internal.cuh"
#include "staged_rows.cuh"

namespace famst {
namespace {

using namespace staged;

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

// Shared memory of one warp: a staged round of 32 rows, the round's
// (eb, n2) and ids, eight task slots.
template <int NKS>
struct Stage : StageRows<NKS> {
    static constexpr int WARPS = NKS >= 16 ? 4 : 8;
    static constexpr int WARP_BYTES = StageRows<NKS>::ROWS_BYTES + 32 * 8 + 32 * 4 + 8 * 16 + 8 * 8;
    static constexpr int SMEM = WARPS * WARP_BYTES;
};

// --------------------------------------------------- per-edge scan (tail)

// argmin over G[c] of (w(c', fixed), 1 + c') with the incumbent (w0, 0).
template <int NKS, int XR>
__device__ __forceinline__ uint64_t scan_staged(
    const float *__restrict__ X, int d, int c, int fixed, float w0, const GLists &g,
    const __nv_bfloat16 *__restrict__ H, const float *__restrict__ heb,
    const float *__restrict__ hn2, uint32_t sbuf, int lane, float aerr, float eps,
    unsigned &evals, unsigned &canon) {
    using S = Stage<NKS>;
    const __nv_bfloat16 *hf = H + int64_t(fixed) * S::LD;
    // B column 0 = the fixed row (lanes 0-3 carry k pairs (2t, 2t+1) and
    // (8+2t, 9+2t) of each k step), columns 1-7 zero
    uint32_t b0[NKS], b1[NKS];
#pragma unroll
    for (int ks = 0; ks < NKS; ++ks) {
        b0[ks] = lane < 4 ? ldg_u32(hf + 16 * ks + 2 * lane) : 0u;
        b1[ks] = lane < 4 ? ldg_u32(hf + 16 * ks + 8 + 2 * lane) : 0u;
    }
    const float ebx = __ldg(heb + fixed), nx = __ldg(hn2 + fixed);
    uint64_t best = uint64_t(__float_as_uint(w0)) << 32;
    const int base = g.off[c], deg = g.off[c + 1] - base;
    const float inf = __int_as_float(0x7f800000);
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
        if (lane == 0) evals += unsigned(__popc(vm));   // every candidate is staged once
        stage_rows<NKS>(H, cand, sbuf, lane);
        float acc[2][4];
        round_dots<NKS>(sbuf, b0, b1, lane, acc);
        __syncwarp();   // every lane's ldmatrix is done before the next round's copies
        // D column 0: lane 4 g holds rows g (acc[.][0]) and g + 8 (acc[.][2]);
        // candidate j = 16 T + r comes from lane 4 (r mod 8)
        const int src = 4 * (lane & 7);
        const float v00 = __shfl_sync(0xffffffffu, acc[0][0], src);
        const float v02 = __shfl_sync(0xffffffffu, acc[0][2], src);
        const float v10 = __shfl_sync(0xffffffffu, acc[1][0], src);
        const float v12 = __shfl_sync(0xffffffffu, acc[1][2], src);
        const float dt = lane < 16 ? ((lane & 8) ? v02 : v00) : ((lane & 8) ? v12 : v10);
        float lo = inf, hi = inf;
        if (valid) dist_bounds(dt, nx, en.y, ebx, en.x, aerr, eps, lo, hi);
        float mh = hi;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) mh = fminf(mh, __shfl_xor_sync(0xffffffffu, mh, o));
        const float bound = __fmul_ru(fminf(mh, key_w(best)), 1.0f + 0x1p-22f);
        unsigned sv = __ballot_sync(0xffffffffu, valid && lo <= bound);
        if (lane == 0) canon += unsigned(__popc(sv));
        while (sv) {   // survivors: canonical distance by the whole warp
            const int sl = __ffs(sv) - 1;
            sv &= sv - 1;
            const int c2 = __shfl_sync(0xffffffffu, cand, sl);
            const uint64_t key = cand_key(canon_w<XR>(X, d, fixed, c2, lane), c2);
            best = key < best ? key : best;
        }
    }
    return best;
}

// Edges handed out one at a time from `order` (its first m entries; NULL:
// 0 .. m-1), each iterated to its own fixed point; change_hist[c] counts the
// edges that changed c times here. A v-scan that repeats the previous
// sweep's inputs is reused.
template <int NKS, int XR, int MINB>
__global__ void __launch_bounds__(Stage<NKS>::WARPS * 32, MINB)
    refine_staged_kernel(const float *__restrict__ X, int d, GLists g,
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
    const uint32_t sbuf = smem_addr(smem + warp * S::WARP_BYTES);
    unsigned long long evals_total = 0, canon_total = 0, scans_total = 0;
    while (true) {
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
            const uint64_t bu = scan_staged<NKS, XR>(X, d, u, v, wt, g, H, heb, hn2, sbuf, lane,
                                                     aerr, eps, evals, canon);
            ++scans_total;
            const int us = key_lo(bu) ? int(key_lo(bu)) - 1 : u;
            float ws = key_w(bu);
            // v-loop: v' in G[v] against the new u*
            uint64_t bv;
            if (v == mv_v && us == mv_u)
                bv = mv_b;
            else {
                bv = scan_staged<NKS, XR>(X, d, v, us, ws, g, H, heb, hn2, sbuf, lane, aerr, eps,
                                          evals, canon);
                ++scans_total;
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
    if (evals_out && lane == 0) {   // pairs, canonical evaluations, rows staged, fixed rows read
        atomicAdd(evals_out, evals_total);
        atomicAdd(evals_out + 1, canon_total);
        atomicAdd(evals_out + 2, evals_total);
        atomicAdd(evals_out + 3, scans_total);
    }
}

// ------------------------------------------- sweep-synchronous phases

// A phase is the u-scans (side 0: c = eu[e], fixed = ev[e]) or the v-scans
// (side 1: c = ev[e], fixed = eu[e]) of the edges list[0 .. *nt).
__global__ void bsp_iota_kernel(int32_t *__restrict__ list, int64_t m) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) list[i] = int32_t(i);
}

__global__ void bsp_count_kernel(const int32_t *__restrict__ list, const int32_t *__restrict__ nt,
                                 int side, const int32_t *__restrict__ eu,
                                 const int32_t *__restrict__ ev, int32_t *__restrict__ cnt,
                                 int32_t *__restrict__ slot) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= *nt) return;
    const int32_t e = list[i];
    const int32_t c = side ? ev[e] : eu[e];
    slot[e] = atomicAdd(&cnt[c], 1);
}

// The scans sorted by scanned vertex, one record per sorted position:
// (edge, fixed point, its eb, its ||h||^2), and the best key starting at the
// edge's incumbent (w, 0).
__global__ void bsp_scatter_kernel(const int32_t *__restrict__ list, const int32_t *__restrict__ nt,
                                   int side, const int32_t *__restrict__ eu,
                                   const int32_t *__restrict__ ev, const float *__restrict__ ew,
                                   const float *__restrict__ heb, const float *__restrict__ hn2,
                                   const int32_t *__restrict__ bstart,
                                   const int32_t *__restrict__ slot, int4 *__restrict__ rec,
                                   unsigned long long *__restrict__ best) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= *nt) return;
    const int32_t e = list[i];
    const int32_t c = side ? ev[e] : eu[e];
    const int32_t fx = side ? eu[e] : ev[e];
    const int64_t pos = int64_t(bstart[c]) + slot[e];
    rec[pos] = make_int4(e, fx, __float_as_int(heb[fx]), __float_as_int(hn2[fx]));
    best[pos] = uint64_t(__float_as_uint(ew[e])) << 32;
}

// Up to four canonical distances (X rows fx[j], c2[j]) computed together,
// each keyed (w, 1 + c2) into sbest[tj] when smaller; warp-uniform inputs.
template <int XR>
__device__ __forceinline__ void canon_batch(const float *__restrict__ X, int d, int nq,
                                            const int (&fx)[4], const int (&c2)[4],
                                            const int (&tj)[4], unsigned long long *sbest,
                                            int lane) {
    if constexpr (XR > 0) {
        float xa[4][XR], xb[4][XR];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < XR; ++q) {
                const int t = lane + 32 * q;
                const bool ok = j < nq && t < d;
                xa[j][q] = ok ? __ldg(X + int64_t(fx[j]) * d + t) : 0.0f;
                xb[j][q] = ok ? __ldg(X + int64_t(c2[j]) * d + t) : 0.0f;
            }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= nq) break;
            float p = 0.0f;
#pragma unroll
            for (int q = 0; q < XR; ++q) {
                const float dl = __fsub_rn(xb[j][q], xa[j][q]);
                p = __fmaf_rn(dl, dl, p);
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
            const uint64_t key = cand_key(__fsqrt_rn(p), c2[j]);
            if (lane == 0 && key < sbest[tj[j]]) sbest[tj[j]] = key;
        }
    } else {
        for (int j = 0; j < nq; ++j) {
            const uint64_t key = cand_key(canon_w<0>(X, d, fx[j], c2[j], lane), c2[j]);
            if (lane == 0 && key < sbest[tj[j]]) sbest[tj[j]] = key;
        }
    }
    __syncwarp();
}

// One warp per scanned vertex c (visited in component order, 32 vertices
// looked up per step): G[c]'s rows are staged once per round of 32 and
// scored against the fixed points of all scans of c, eight per mma; the
// best key of the scan at sorted position i is kept in best[i].
template <int NKS, int XR, int MINB>
__global__ void __launch_bounds__(Stage<NKS>::WARPS * 32, MINB)
    refine_group_kernel(const float *__restrict__ X, int d, GLists g,
                        const __nv_bfloat16 *__restrict__ H, const int32_t *__restrict__ members,
                        int64_t n, const int32_t *__restrict__ bstart,
                        const int4 *__restrict__ rec, unsigned long long *__restrict__ best,
                        unsigned long long *__restrict__ evals_out, float aerr, float eps) {
    using S = Stage<NKS>;
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    char *wb = smem + warp * S::WARP_BYTES;
    const uint32_t sbuf = smem_addr(wb);
    float2 *s_en = reinterpret_cast<float2 *>(wb + S::ROWS_BYTES);           // 32 (eb, n2)
    int32_t *s_id = reinterpret_cast<int32_t *>(wb + S::ROWS_BYTES + 256);   // 32 ids
    float4 *s_task = reinterpret_cast<float4 *>(wb + S::ROWS_BYTES + 384);   // 8 (fixed, eb, n2)
    unsigned long long *s_best =
        reinterpret_cast<unsigned long long *>(wb + S::ROWS_BYTES + 512);    // 8 best keys
    const float inf = __int_as_float(0x7f800000);
    const int g4 = lane >> 2, t4 = lane & 3;   // mma fragment row group / column pair
    // counters, one per lane: pairs (lane 0), canonical evaluations (1),
    // rows staged (2), fixed rows read (3)
    unsigned long long ctr = 0;
    // warp w visits the members at w, w + W, w + 2W, ... (W warps in all),
    // so the warps work on neighbouring members, i.e. a few components at a
    // time; the next 32 of its vertices are looked up together
    const int64_t nw = int64_t(gridDim.x) * S::WARPS;
    const int64_t w0 = int64_t(blockIdx.x) * S::WARPS + warp;
    for (int64_t p0 = w0; p0 < n; p0 += 32 * nw) {
        int cl = 0, tl0 = 0, tl1 = 0, gl0 = 0, gl1 = 0;
        const int64_t pl = p0 + int64_t(lane) * nw;
        if (pl < n) {
            cl = members[pl];
            tl0 = bstart[cl];
            tl1 = bstart[cl + 1];
            if (tl1 > tl0) {
                gl0 = g.off[cl];
                gl1 = g.off[cl + 1];
            }
        }
        unsigned busy = __ballot_sync(0xffffffffu, tl1 > tl0);
        while (busy) {
            const int src = __ffs(busy) - 1;
            busy &= busy - 1;
            const int t0 = __shfl_sync(0xffffffffu, tl0, src);
            const int t1 = __shfl_sync(0xffffffffu, tl1, src);
            const int base = __shfl_sync(0xffffffffu, gl0, src);
            const int deg = __shfl_sync(0xffffffffu, gl1, src) - base;
            // a vertex with at most eight scans loads its task block (records
            // and best keys, in shared memory) once for all its rounds
            const bool single = t1 - t0 <= 8;
            for (int r0 = 0; r0 < deg; r0 += 32) {
                const int idx = r0 + lane;
                const bool valid = idx < deg;
                int cand = -1;
                float2 en = make_float2(inf, 0.0f);
                if (valid) {
                    cand = __ldg(g.id + base + idx);
                    en = __ldg(g.en + base + idx);
                }
                const int nv = __popc(__ballot_sync(0xffffffffu, valid));
                s_en[lane] = en;
                s_id[lane] = cand;
                stage_rows<NKS>(H, cand, sbuf, lane);
                if (lane == 2) ctr += unsigned(nv);
                for (int tb = t0; tb < t1; tb += 8) {
                    const int ntb = t1 - tb < 8 ? t1 - tb : 8;
                    if (!single || r0 == 0) {
                        if (lane < ntb) {
                            const int4 r = rec[tb + lane];
                            s_task[lane] = make_float4(__int_as_float(r.y), __int_as_float(r.z),
                                                       __int_as_float(r.w), 0.0f);
                            s_best[lane] = best[tb + lane];
                        }
                        __syncwarp();
                    }
                    if (lane == 3) ctr += unsigned(ntb);
                    // B column j = the fixed row of task slot j (lane 4 j + t
                    // carries k pairs (2t, 2t+1) and (8+2t, 9+2t) of each k step)
                    uint32_t b0[NKS], b1[NKS];
                    {
                        const bool has = g4 < ntb;
                        const __nv_bfloat16 *hf =
                            H + int64_t(has ? __float_as_int(s_task[g4].x) : 0) * S::LD;
#pragma unroll
                        for (int ks = 0; ks < NKS; ++ks) {
                            b0[ks] = has ? ldg_u32(hf + 16 * ks + 2 * t4) : 0u;
                            b1[ks] = has ? ldg_u32(hf + 16 * ks + 8 + 2 * t4) : 0u;
                        }
                    }
                    float acc[2][4];
                    round_dots<NKS>(sbuf, b0, b1, lane, acc);
                    // this lane holds the pairs (candidate 16 T + g4 + 8 (e2 >> 1),
                    // task 2 t4 + (e2 & 1)) in acc[T][e2]
                    float lo[2][4];
                    float mh0 = inf, mh1 = inf;
#pragma unroll
                    for (int T = 0; T < 2; ++T)
#pragma unroll
                        for (int e2 = 0; e2 < 4; ++e2) {
                            const int ci = 16 * T + g4 + 8 * (e2 >> 1), tj = 2 * t4 + (e2 & 1);
                            float hi = inf;
                            lo[T][e2] = inf;
                            if (ci < nv && tj < ntb) {
                                const float2 ce = s_en[ci];
                                const float4 ts = s_task[tj];
                                dist_bounds(acc[T][e2], ts.z, ce.y, ts.y, ce.x, aerr, eps,
                                            lo[T][e2], hi);
                            }
                            if (e2 & 1) mh1 = fminf(mh1, hi);
                            else mh0 = fminf(mh0, hi);
                        }
                    // per task: the smallest upper bound over all candidates
                    // (the lanes with the same t4)
#pragma unroll
                    for (int o = 4; o <= 16; o <<= 1) {
                        mh0 = fminf(mh0, __shfl_xor_sync(0xffffffffu, mh0, o));
                        mh1 = fminf(mh1, __shfl_xor_sync(0xffffffffu, mh1, o));
                    }
                    const float bnd0 =
                        2 * t4 < ntb
                            ? __fmul_ru(fminf(mh0, key_w(s_best[2 * t4])), 1.0f + 0x1p-22f)
                            : -inf;
                    const float bnd1 =
                        2 * t4 + 1 < ntb
                            ? __fmul_ru(fminf(mh1, key_w(s_best[2 * t4 + 1])), 1.0f + 0x1p-22f)
                            : -inf;
                    if (lane == 0) ctr += unsigned(nv * ntb);
                    __syncwarp();
                    // survivors, decided on canonical distances by the whole
                    // warp, up to four at a time; bit 4 T + e2 of `my` marks a
                    // surviving pair of this lane (one copy of the batch code).
                    unsigned my = 0;
#pragma unroll
                    for (int T = 0; T < 2; ++T)
#pragma unroll
                        for (int e2 = 0; e2 < 4; ++e2)
                            if (16 * T + g4 + 8 * (e2 >> 1) < nv && 2 * t4 + (e2 & 1) < ntb &&
                                lo[T][e2] <= ((e2 & 1) ? bnd1 : bnd0))
                                my |= 1u << (4 * T + e2);
                    {
                        int cnt = __popc(my);
#pragma unroll
                        for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                        if (lane == 1) ctr += unsigned(cnt);
                    }
#pragma unroll 1
                    while (true) {
                        int qf[4], qc[4], qt[4], nq = 0;
#pragma unroll 1
                        while (nq < 4) {
                            const unsigned any = __ballot_sync(0xffffffffu, my != 0u);
                            if (!any) break;
                            const int sl = __ffs(any) - 1;
                            const int bit = __ffs(__shfl_sync(0xffffffffu, my, sl)) - 1;
                            if (lane == sl) my &= my - 1u;
                            const int ci = 16 * (bit >> 2) + (sl >> 2) + 8 * ((bit & 3) >> 1);
                            const int tj = 2 * (sl & 3) + (bit & 1);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (j == nq) {
                                    qc[j] = s_id[ci];
                                    qf[j] = __float_as_int(s_task[tj].x);
                                    qt[j] = tj;
                                }
                            ++nq;
                        }
                        if (nq == 0) break;
                        canon_batch<XR>(X, d, nq, qf, qc, qt, s_best, lane);
                    }
                    if ((!single || r0 + 32 >= deg) && lane < ntb) best[tb + lane] = s_best[lane];
                    __syncwarp();
                }
                __syncwarp();   // the rows stay until every task block is done
            }
        }
    }
    if (evals_out && lane < 4) atomicAdd(evals_out + lane, ctr);
}

// After the u-scans: move u; an edge whose u stays and whose v did not move
// in the previous sweep is at its fixed point (its v-scan would repeat the
// previous one); the others go on to the v-scans.
__global__ void bsp_finish_u_kernel(const int32_t *__restrict__ list, const int32_t *__restrict__ nt,
                                    int32_t *__restrict__ eu, float *__restrict__ ew,
                                    const int32_t *__restrict__ bstart,
                                    const int32_t *__restrict__ slot,
                                    const unsigned long long *__restrict__ best,
                                    const uint8_t *__restrict__ vstable, uint8_t *__restrict__ uchg,
                                    int32_t *__restrict__ listB, int32_t *__restrict__ nB,
                                    int32_t *__restrict__ hist, int sweep) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= *nt) return;
    const int32_t e = list[i];
    const unsigned long long b = best[int64_t(bstart[eu[e]]) + slot[e]];
    const bool moved = key_lo(b) != 0;
    if (moved) eu[e] = int32_t(key_lo(b)) - 1;
    ew[e] = key_w(b);
    uchg[e] = moved ? 1 : 0;
    if (!moved && vstable[e]) {
        atomicAdd(&hist[sweep], 1);   // unchanged in this sweep: converged
        return;
    }
    listB[atomicAdd(nB, 1)] = e;
}

// After the v-scans: move v; changed edges stay active for the next sweep.
__global__ void bsp_finish_v_kernel(const int32_t *__restrict__ listB, const int32_t *__restrict__ nB,
                                    int32_t *__restrict__ ev, float *__restrict__ ew,
                                    const int32_t *__restrict__ bstart,
                                    const int32_t *__restrict__ slot,
                                    const unsigned long long *__restrict__ best,
                                    uint8_t *__restrict__ vstable, const uint8_t *__restrict__ uchg,
                                    int32_t *__restrict__ next, int32_t *__restrict__ nnext,
                                    int32_t *__restrict__ hist, int sweep) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= *nB) return;
    const int32_t e = listB[i];
    const unsigned long long b = best[int64_t(bstart[ev[e]]) + slot[e]];
    const bool moved = key_lo(b) != 0;
    if (moved) ev[e] = int32_t(key_lo(b)) - 1;
    ew[e] = key_w(b);
    vstable[e] = moved ? 0 : 1;
    if (moved || uchg[e]) {
        next[atomicAdd(nnext, 1)] = e;
    } else {
        atomicAdd(&hist[sweep], 1);
    }
}

// |p~ - ||h_x - h_y||^2| <= aerr (||h_x||^2 + ||h_y||^2) + 1e-35: the BF16
// products are exact in FP32; an accumulation that aligns each block of 16
// products (plus the running sum) to its largest exponent and keeps 24 bits
// loses at most 17 2^-23 of the block's absolute sum, about
// ld 2^-23 (||h_x||^2 + ||h_y||^2) over the row for 2 h_x.h_y. It is taken 16
// times over (an accumulator keeping only 20 bits would still be covered),
// plus the norms' and the two final roundings; 1e-35 covers products flushed
// below the FP32 normal range.
template <int NKS>
float refine_aerr() {
    return float(Stage<NKS>::LD * std::ldexp(1.0, -19) + std::ldexp(1.0, -20));
}

// canonical distance vs the exact one, generously: (d + 16) u
float refine_eps(int d) { return float((d + 16) * std::ldexp(1.0, -24) * 1.1); }

template <class K>
famst_status occupancy_grid(const Exec &ex, K *fn, int threads, int smem, int64_t want,
                            unsigned *grid) {
    if (set_smem_attr(fn, smem, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t cap = int64_t(ex.num_sms) * per_sm;
    *grid = unsigned(want < cap ? (want > 0 ? want : 1) : cap);
    return FAMST_OK;
}

template <int NKS, int XR, int MINB>
famst_status launch_staged_t(const Exec &ex, const float *X, int d, const HalfRows &hr,
                             int32_t *eu, int32_t *ev, float *ew, const int32_t *order, int64_t m,
                             int max_iters, int32_t *change_hist, unsigned long long *next_item,
                             unsigned long long *evals) {
    using S = Stage<NKS>;
    unsigned grid;
    auto *fn = refine_staged_kernel<NKS, XR, MINB>;
    famst_status st =
        occupancy_grid(ex, fn, S::WARPS * 32, S::SMEM, (m + S::WARPS - 1) / S::WARPS, &grid);
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, fn, grid, S::WARPS * 32, S::SMEM, X, d, hr.g, hr.h, hr.eb, hr.n2, eu, ev, ew,
                 order, m, max_iters, change_hist, next_item, ex.dstatus, evals,
                 refine_aerr<NKS>(), refine_eps(d));
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

template <int NKS, int XR, int MINB>
famst_status launch_group_t(const Exec &ex, const float *X, int d, const HalfRows &hr,
                            const int32_t *members, int64_t n, const int32_t *bstart,
                            const int4 *rec, unsigned long long *best, unsigned long long *evals) {
    using S = Stage<NKS>;
    unsigned grid;
    auto *fn = refine_group_kernel<NKS, XR, MINB>;
    famst_status st =
        occupancy_grid(ex, fn, S::WARPS * 32, S::SMEM, (n + S::WARPS - 1) / S::WARPS, &grid);
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, fn, grid, S::WARPS * 32, S::SMEM, X, d, hr.g, hr.h, members, n, bstart, rec,
                 best, evals, refine_aerr<NKS>(), refine_eps(d));
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

famst_status launch_group(const Exec &ex, const float *X, int d, const HalfRows &hr,
                          const int32_t *members, int64_t n, const int32_t *bstart,
                          const int4 *rec, unsigned long long *best, unsigned long long *evals) {
    if (hr.ld == 64)
        return launch_group_t<4, 2, 4>(ex, X, d, hr, members, n, bstart, rec, best, evals);
    if (hr.ld == 128)
        return launch_group_t<8, 4, 3>(ex, X, d, hr, members, n, bstart, rec, best, evals);
    return launch_group_t<16, 0, 2>(ex, X, d, hr, members, n, bstart, rec, best, evals);
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

bool refine_staged_supported(const HalfRows &hr) {
    return hr.h && hr.g.id && (hr.ld == 64 || hr.ld == 128 || hr.ld == 256);
}

famst_status launch_refine_staged(const Exec &ex, const float *X, int d, const HalfRows &hr,
                                  int32_t *eu, int32_t *ev, float *ew, const int32_t *order,
                                  int64_t m, int max_iters, int32_t *change_hist,
                                  unsigned long long *next_item, unsigned long long *evals) {
    if (hr.ld == 64)
        return launch_staged_t<4, 2, 4>(ex, X, d, hr, eu, ev, ew, order, m, max_iters, change_hist,
                                        next_item, evals);
    if (hr.ld == 128)
        return launch_staged_t<8, 4, 3>(ex, X, d, hr, eu, ev, ew, order, m, max_iters, change_hist,
                                        next_item, evals);
    return launch_staged_t<16, 0, 2>(ex, X, d, hr, eu, ev, ew, order, m, max_iters, change_hist,
                                     next_item, evals);
}

size_t refine_build_workspace(int64_t n, int64_t m) {
    return 2 * align256(size_t(n + 1) * 4) + scan_workspace(n + 1) + 3 * align256(size_t(m) * 4) +
           align256(size_t(m) * 16) + align256(size_t(m) * 8) + 2 * align256(size_t(m)) +
           align256(64);
}

// Algorithm 4 repeated until no edge changes (Algorithm 1), inside a build:
// sweeps run sweep-synchronously while more than m / 16 edges are active,
// then the remaining active edges run per edge. change_hist[c] receives the
// number of edges that changed in exactly c sweeps (the bookkeeping of
// refine_edges); pinned_host: two pinned host words.
famst_status refine_build(const Exec &ex, Arena &ar, const float *X, int d, const HalfRows &hr,
                          const int32_t *members, int64_t n, int32_t *eu, int32_t *ev, float *ew,
                          const int32_t *order, int64_t m, int max_iters, int32_t *change_hist,
                          unsigned long long *evals, int32_t *pinned_host) {
    if (m == 0) return FAMST_OK;
    int32_t *cnt = ar.take<int32_t>(size_t(n + 1));
    int32_t *bstart = ar.take<int32_t>(size_t(n + 1));
    int32_t *slot = ar.take<int32_t>(size_t(m));
    int4 *rec = ar.take<int4>(size_t(m));
    int32_t *listA = ar.take<int32_t>(size_t(m));
    int32_t *listB = ar.take<int32_t>(size_t(m));
    unsigned long long *best = ar.take<unsigned long long>(size_t(m));
    uint8_t *vstable = ar.take<uint8_t>(size_t(m));
    uint8_t *uchg = ar.take<uint8_t>(size_t(m));
    int32_t *counts = ar.take<int32_t>(16);   // [0] |list A|, [1] |list B|, [2] next; [8..9] cursor
    if (!cnt || !bstart || !slot || !rec || !listA || !listB || !best || !vstable || !uchg ||
        !counts)
        return FAMST_ERR_OOM;
    unsigned long long *next_item = reinterpret_cast<unsigned long long *>(counts + 8);
    if (cudaMemsetAsync(vstable, 0, size_t(m), ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    const int th = 256;
    auto blocks = [](int64_t c) { return unsigned((c + 255) / 256); };
    auto phase = [&](const int32_t *list, const int32_t *nt, int64_t nmax,
                     int side) -> famst_status {
        if (cudaMemsetAsync(cnt, 0, size_t(n + 1) * 4, ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        FAMST_LAUNCH(ex, bsp_count_kernel, blocks(nmax), th, 0, list, nt, side, eu, ev, cnt, slot);
        const size_t mark = ar.off;   // the scan's scratch is reused by every phase
        famst_status st = exclusive_scan_i32(ex, ar, cnt, bstart, n + 1, nullptr);
        ar.off = mark;
        if (st != FAMST_OK) return st;
        FAMST_LAUNCH(ex, bsp_scatter_kernel, blocks(nmax), th, 0, list, nt, side, eu, ev, ew, hr.eb,
                     hr.n2, bstart, slot, rec, best);
        return launch_group(ex, X, d, hr, members, n, bstart, rec, best, evals);
    };
    timer_mark(ex, TIMER_REFINE, false);
    FAMST_LAUNCH(ex, bsp_iota_kernel, blocks(m), th, 0, listA, m);
    int64_t active = m;
    int sweep = 0;
    const int64_t tail_at = m / 16;
    // sweep-synchronous sweeps (none when max_iters == 1: the per-edge kernel
    // then applies the cap)
    while (active > tail_at && sweep < max_iters - 1) {
        pinned_host[0] = int32_t(active);
        if (cudaMemcpyAsync(counts, pinned_host, 4, cudaMemcpyHostToDevice, ex.stream) !=
                cudaSuccess ||
            cudaMemsetAsync(counts + 1, 0, 8, ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        famst_status st = phase(listA, counts, active, 0);
        if (st != FAMST_OK) return st;
        FAMST_LAUNCH(ex, bsp_finish_u_kernel, blocks(active), th, 0, listA, counts, eu, ew, bstart,
                     slot, best, vstable, uchg, listB, counts + 1, change_hist, sweep);
        st = phase(listB, counts + 1, active, 1);
        if (st != FAMST_OK) return st;
        // listA receives the edges still active (count in counts[2])
        FAMST_LAUNCH(ex, bsp_finish_v_kernel, blocks(active), th, 0, listB, counts + 1, ev, ew,
                     bstart, slot, best, vstable, uchg, listA, counts + 2, change_hist, sweep);
        if (cudaMemcpyAsync(pinned_host + 1, counts + 2, 4, cudaMemcpyDeviceToHost, ex.stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        active = pinned_host[1];
        ++sweep;
    }
    // the remaining active edges, each to its own fixed point; their change
    // counts continue from `sweep`
    if (active > 0) {
        if (cudaMemsetAsync(next_item, 0, 8, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
        famst_status st = launch_refine_staged(ex, X, d, hr, eu, ev, ew, sweep == 0 ? order : listA,
                                               active, max_iters - sweep, change_hist + sweep,
                                               next_item, evals);
        if (st != FAMST_OK) return st;
    }
    timer_mark(ex, TIMER_REFINE, true);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst
