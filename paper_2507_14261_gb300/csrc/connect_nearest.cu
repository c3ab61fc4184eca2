// The nearest-pair variant of Algorithm 3: for every component pair i < j,
// the lambda pairs (u in C_i, v in C_j) with the smallest canonical distance
// under the edge order (w, min id, max id) -- "the lambda nearest
// cross-component edges" -- instead of the lambda shortest of lambda^2
// random samples. A component pair with fewer than lambda cross pairs
// repeats its farthest pair in the remaining slots.
//
// The work is all cross pairs, |C_i| |C_j| per component pair (n^2 / 2 over
// all pairs when the components cover the points), so it is organised like
// a GEMM over the points sorted by component:
//  * a work item is a block of 32 consecutive members of one component C_i;
//    its warp stages their centred BF16 rows in shared memory once and then
//    streams the members of every later component C_j (j > i), eight per
//    step, as the B columns of mma.sync m16n8k16 (32 x 8 dot products per
//    k chunk), reading each row's error bound and norm alongside;
//  * rigorous bounds on the canonical distance (staged_rows.cuh) rule pairs
//    out against the warp's current lambda-th best (before lambda pairs are
//    known: the lambda-th smallest upper bound of the step), survivors are
//    decided on canonical FP32 distances four at a time, and the warp keeps
//    a sorted top-lambda list of (w, min id, max id) keys, one entry per
//    lane, for each (item, C_j);
//  * a second kernel merges, per component pair, the lists of its C_i
//    blocks into the final lambda edges, written in Algorithm 3's layout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "famst_internal.cuh"
#include "staged_rows.cuh"

namespace famst {
namespace {

using namespace staged;

constexpr int NP_WARPS = 4;   // warps per block

template <int NKS>
struct NpStage : StageRows<NKS> {
    // per warp: the block's rows, their (eb, n2) and ids, the step's eight
    // (id, eb, n2) of the B columns
    static constexpr int WARP_BYTES = StageRows<NKS>::ROWS_BYTES + 32 * 8 + 32 * 4 + 8 * 16;
    static constexpr int SMEM = NP_WARPS * WARP_BYTES;
};

// (w, min id, max id) as two words: hi = w bits << 32 | min id, lo = max id
__device__ __forceinline__ bool pkey_less(uint64_t ah, uint32_t al, uint64_t bh, uint32_t bl) {
    return ah < bh || (ah == bh && al < bl);
}
__device__ __forceinline__ uint64_t pkey_hi(float w, int a, int b) {
    return (uint64_t(__float_as_uint(w)) << 32) | uint32_t(a < b ? a : b);
}

// Insert (kh, kl, u, v) into the warp's sorted list (lane r holds entry r,
// entries beyond `have` hold +inf keys); warp-uniform arguments.
__device__ __forceinline__ void list_insert(uint64_t &eh, uint32_t &el, int &eu, int &ev,
                                            uint64_t kh, uint32_t kl, int u, int v, int lambda,
                                            int &have, int lane) {
    const unsigned before = __ballot_sync(0xffffffffu, lane < have && pkey_less(eh, el, kh, kl));
    const int pos = __popc(before);
    if (pos >= lambda) return;
    const uint64_t ph = shfl_up_u64(eh, 1);
    const uint32_t pl = __shfl_up_sync(0xffffffffu, el, 1);
    const int pu = __shfl_up_sync(0xffffffffu, eu, 1);
    const int pv = __shfl_up_sync(0xffffffffu, ev, 1);
    if (lane > pos && lane < lambda) {
        eh = ph;
        el = pl;
        eu = pu;
        ev = pv;
    } else if (lane == pos) {
        eh = kh;
        el = kl;
        eu = u;
        ev = v;
    }
    if (have < lambda) ++have;
}

// Up to four canonical distances of pairs (ua[j], vb[j]) computed together
// and inserted into the list.
template <int XR>
__device__ __forceinline__ void pairs_batch(const float *__restrict__ X, int d, int nq,
                                            const int (&ua)[4], const int (&vb)[4],
                                            uint64_t &eh, uint32_t &el, int &eu, int &ev,
                                            int lambda, int &have, int lane) {
    if constexpr (XR > 0) {
        float xa[4][XR], xb[4][XR];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < XR; ++q) {
                const int t = lane + 32 * q;
                const bool ok = j < nq && t < d;
                xa[j][q] = ok ? __ldg(X + int64_t(ua[j]) * d + t) : 0.0f;
                xb[j][q] = ok ? __ldg(X + int64_t(vb[j]) * d + t) : 0.0f;
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
            const float w = __fsqrt_rn(p);
            const int a = ua[j], b = vb[j];
            list_insert(eh, el, eu, ev, pkey_hi(w, a, b), uint32_t(a < b ? b : a), a, b, lambda,
                        have, lane);
        }
    } else {
        for (int j = 0; j < nq; ++j) {
            const float w = canon_w<0>(X, d, ua[j], vb[j], lane);
            const int a = ua[j], b = vb[j];
            list_insert(eh, el, eu, ev, pkey_hi(w, a, b), uint32_t(a < b ? b : a), a, b, lambda,
                        have, lane);
        }
    }
}

// One warp per work item (component i, block of 32 of its members): the
// top-lambda list of every later component j goes to out[(item, j - i - 1)].
// item_off[i] = first item of component i (t + 1 entries), out_off[i] =
// first output slot (in lists) of component i's items.
template <int NKS, int XR>
__global__ void __launch_bounds__(NP_WARPS * 32)
    nearest_pairs_kernel(const float *__restrict__ X, int d, const __nv_bfloat16 *__restrict__ H,
                         const float *__restrict__ heb, const float *__restrict__ hn2,
                         const int32_t *__restrict__ members, const int32_t *__restrict__ comp_off,
                         const int64_t *__restrict__ item_off, const int64_t *__restrict__ out_off,
                         int64_t t, int64_t items, int lambda, int32_t *__restrict__ ou,
                         int32_t *__restrict__ ov, float *__restrict__ ow, float aerr, float eps,
                         unsigned long long *__restrict__ stats) {
    using S = NpStage<NKS>;
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    char *wb = smem + warp * S::WARP_BYTES;
    const uint32_t sbuf = smem_addr(wb);
    float2 *s_en = reinterpret_cast<float2 *>(wb + S::ROWS_BYTES);          // 32 (eb, n2) of u
    int32_t *s_u = reinterpret_cast<int32_t *>(wb + S::ROWS_BYTES + 256);   // 32 ids of u
    float4 *s_v = reinterpret_cast<float4 *>(wb + S::ROWS_BYTES + 384);     // 8 (id, eb, n2) of v
    const float inf = __int_as_float(0x7f800000);
    const int g4 = lane >> 2, t4 = lane & 3;
    unsigned long long pairs = 0, canon = 0;
    const int64_t nw = int64_t(gridDim.x) * NP_WARPS;
    for (int64_t q = int64_t(blockIdx.x) * NP_WARPS + warp; q < items; q += nw) {
        // component i of item q: the last i with item_off[i] <= q
        int64_t lo_i = 0, hi_i = t;   // item_off[lo_i] <= q < item_off[hi_i]
        while (hi_i - lo_i > 1) {
            const int64_t mid = (lo_i + hi_i) >> 1;
            if (item_off[mid] <= q) lo_i = mid; else hi_i = mid;
        }
        const int64_t i = lo_i;
        const int64_t b = q - item_off[i];
        const int u0 = comp_off[i] + int(b) * 32;
        const int nu = min(32, comp_off[i + 1] - u0);
        int myu = -1;
        float2 ue = make_float2(inf, 0.0f);
        if (lane < nu) {
            myu = members[u0 + lane];
            ue = make_float2(__ldg(heb + myu), __ldg(hn2 + myu));
        }
        s_en[lane] = ue;
        s_u[lane] = myu;
        stage_rows<NKS>(H, myu, sbuf, lane);
        int64_t slot = out_off[i] + b * (t - 1 - i);
        for (int64_t j = i + 1; j < t; ++j, ++slot) {
            uint64_t eh = ~0ull;
            uint32_t el = ~0u;
            int eu = -1, ev = -1, have = 0;
            const int v0 = comp_off[j], v1 = comp_off[j + 1];
            for (int vc = v0; vc < v1; vc += 8) {
                const int nvb = min(8, v1 - vc);
                if (lane < nvb) {
                    const int v = members[vc + lane];
                    s_v[lane] = make_float4(__int_as_float(v), __ldg(heb + v), __ldg(hn2 + v), 0.0f);
                }
                __syncwarp();
                uint32_t b0[NKS], b1[NKS];
                {
                    const bool has = g4 < nvb;
                    const __nv_bfloat16 *hf =
                        H + int64_t(has ? __float_as_int(s_v[g4].x) : 0) * S::LD;
#pragma unroll
                    for (int ks = 0; ks < NKS; ++ks) {
                        b0[ks] = has ? ldg_u32(hf + 16 * ks + 2 * t4) : 0u;
                        b1[ks] = has ? ldg_u32(hf + 16 * ks + 8 + 2 * t4) : 0u;
                    }
                }
                float acc[2][4];
                round_dots<NKS>(sbuf, b0, b1, lane, acc);
                // this lane: pairs (u slot 16 T + g4 + 8 (e2 >> 1), v slot 2 t4 + (e2 & 1))
                float lo[2][4], hi[2][4];
#pragma unroll
                for (int T = 0; T < 2; ++T)
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        const int ui = 16 * T + g4 + 8 * (e2 >> 1), vj = 2 * t4 + (e2 & 1);
                        lo[T][e2] = inf;
                        hi[T][e2] = inf;
                        if (ui < nu && vj < nvb) {
                            const float2 a = s_en[ui];
                            const float4 c = s_v[vj];
                            dist_bounds(acc[T][e2], a.y, c.z, a.x, c.y, aerr, eps, lo[T][e2],
                                        hi[T][e2]);
                        }
                    }
                if (lane == 0) pairs += unsigned(nu * nvb);
                // threshold: the list's lambda-th weight; while the list is not
                // full, the lambda-th smallest upper bound of this step (lambda
                // pairs at most that far exist, so a pair above it is beaten)
                float thr = have == lambda ? __uint_as_float(uint32_t(__shfl_sync(
                                                 0xffffffffu, uint32_t(eh >> 32), lambda - 1)))
                                           : inf;
                if (have < lambda) {
                    float hv[8];
#pragma unroll
                    for (int T = 0; T < 2; ++T)
#pragma unroll
                        for (int e2 = 0; e2 < 4; ++e2) hv[4 * T + e2] = hi[T][e2];
                    float kth = inf;
                    for (int r = 0; r < lambda; ++r) {
                        float m = inf;
                        int at = -1;
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (hv[e] < m) {
                                m = hv[e];
                                at = e;
                            }
                        float wm = m;
#pragma unroll
                        for (int o = 16; o >= 1; o >>= 1)
                            wm = fminf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
                        kth = wm;
                        if (!(wm < inf)) break;
                        // remove one occurrence: the lowest lane holding it
                        const unsigned holders = __ballot_sync(0xffffffffu, m == wm && at >= 0);
                        if (lane == __ffs(holders) - 1) {
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                if (e == at) hv[e] = inf;
                        }
                    }
                    thr = fminf(thr, kth);
                }
                const float bound = __fmul_ru(thr, 1.0f + 0x1p-22f);
                // survivors among the valid pairs only (the bound is +inf while a
                // step has fewer than lambda pairs)
                unsigned my = 0;
#pragma unroll
                for (int T = 0; T < 2; ++T)
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        const int ui = 16 * T + g4 + 8 * (e2 >> 1), vj = 2 * t4 + (e2 & 1);
                        if (ui < nu && vj < nvb && lo[T][e2] <= bound) my |= 1u << (4 * T + e2);
                    }
                {
                    int cnt = __popc(my);
#pragma unroll
                    for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                    if (lane == 0) canon += unsigned(cnt);
                }
#pragma unroll 1
                while (true) {
                    int qa[4], qb[4], nq = 0;
#pragma unroll 1
                    while (nq < 4) {
                        const unsigned any = __ballot_sync(0xffffffffu, my != 0u);
                        if (!any) break;
                        const int sl = __ffs(any) - 1;
                        const int bit = __ffs(__shfl_sync(0xffffffffu, my, sl)) - 1;
                        if (lane == sl) my &= my - 1u;
                        const int ui = 16 * (bit >> 2) + (sl >> 2) + 8 * ((bit & 3) >> 1);
                        const int vj = 2 * (sl & 3) + (bit & 1);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (e == nq) {
                                qa[e] = s_u[ui];
                                qb[e] = __float_as_int(s_v[vj].x);
                            }
                        ++nq;
                    }
                    if (nq == 0) break;
                    pairs_batch<XR>(X, d, nq, qa, qb, eh, el, eu, ev, lambda, have, lane);
                }
                __syncwarp();   // s_v is rewritten by the next step
            }
            // the list, padded by repeating its last entry
            const int src = lane < have ? lane : have - 1;
            const int ru = __shfl_sync(0xffffffffu, eu, src);
            const int rv = __shfl_sync(0xffffffffu, ev, src);
            const float rw = __uint_as_float(uint32_t(shfl_idx_u64(eh, src) >> 32));
            if (lane < lambda) {
                ou[slot * lambda + lane] = ru;
                ov[slot * lambda + lane] = rv;
                ow[slot * lambda + lane] = rw;
            }
        }
        __syncwarp();   // the block's rows stay until every component j is done
    }
    if (stats && lane == 0) {
        atomicAdd(stats, pairs);
        atomicAdd(stats + 1, canon);
    }
}

// Per component pair (i, j): merge the lists of C_i's blocks (nb_i lists of
// lambda entries) into the lambda smallest (w, min id, max id), written as
// edges (pair rank) * lambda + r with u in C_i, v in C_j. One warp per pair.
__global__ void nearest_merge_kernel(const int32_t *__restrict__ comp_off,
                                     const int64_t *__restrict__ out_off, int64_t t, int lambda,
                                     const int32_t *__restrict__ ou, const int32_t *__restrict__ ov,
                                     const float *__restrict__ ow, int32_t *__restrict__ eu,
                                     int32_t *__restrict__ ev, float *__restrict__ ew,
                                     int32_t *__restrict__ eci, int32_t *__restrict__ ecj) {
    const int lane = threadIdx.x & 31;
    const int64_t npairs = t * (t - 1) / 2;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t p = w0; p < npairs; p += nw) {
        // pair p -> (i, j), pairs enumerated i outer, j inner
        int64_t i = 0;
        {
            const double bb = 2.0 * double(t) - 1.0;
            const double disc = bb * bb - 8.0 * double(p);
            i = int64_t((bb - sqrt(disc > 0 ? disc : 0.0)) * 0.5);
            if (i < 0) i = 0;
            if (i > t - 2) i = t - 2;
            auto start = [t](int64_t x) { return x * t - x * (x + 1) / 2; };
            while (i > 0 && start(i) > p) --i;
            while (i + 1 <= t - 2 && start(i + 1) <= p) ++i;
        }
        const int64_t j = p - (i * t - i * (i + 1) / 2) + i + 1;
        const int64_t nb = (comp_off[i + 1] - comp_off[i] + 31) / 32;
        const int64_t total = nb * lambda;
        // the lists of this pair sit at out_off[i] + b (t - 1 - i) + (j - i - 1)
        uint64_t bh = ~0ull;
        uint32_t bl = ~0u;
        int bu = -1, bv = -1;
        for (int r = 0; r < lambda; ++r) {
            // the r-th smallest: every lane scans its share, warp minimum
            uint64_t mh = ~0ull;
            uint32_t ml = ~0u;
            int64_t at = -1;
            for (int64_t e = lane; e < total; e += 32) {
                const int64_t b = e / lambda, rr = e - b * lambda;
                const int64_t s = (out_off[i] + b * (t - 1 - i) + (j - i - 1)) * lambda + rr;
                const int a = ou[s], c = ov[s];
                const uint64_t h = pkey_hi(ow[s], a, c);
                const uint32_t l = uint32_t(a < c ? c : a);
                // strictly after the previous pick: a pair sits in one block's
                // list only, so equal keys are a list's padding repeats
                const bool after = r == 0 || pkey_less(bh, bl, h, l);
                if (after && pkey_less(h, l, mh, ml)) {
                    mh = h;
                    ml = l;
                    at = s;
                }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const uint64_t oh = shfl_xor_u64(mh, o);
                const uint32_t ol = __shfl_xor_sync(0xffffffffu, ml, o);
                const int64_t oa = int64_t(shfl_xor_u64(uint64_t(at), o));
                if (pkey_less(oh, ol, mh, ml) || (oh == mh && ol == ml && oa < at)) {
                    mh = oh;
                    ml = ol;
                    at = oa;
                }
            }
            if (at >= 0) {
                bh = mh;
                bl = ml;
                bu = ou[at];
                bv = ov[at];
            }
            // fewer distinct pairs than lambda: repeat the last one
            if (lane == 0) {
                const int64_t e = p * lambda + r;
                eu[e] = bu;
                ev[e] = bv;
                ew[e] = __uint_as_float(uint32_t(bh >> 32));
                eci[e] = int32_t(i);
                ecj[e] = int32_t(j);
            }
        }
    }
}

template <int NKS, int XR>
famst_status launch_np(const Exec &ex, const float *X, int d, const HalfRows &hr,
                       const int32_t *members, const int32_t *comp_off, const int64_t *item_off,
                       const int64_t *out_off, int64_t t, int64_t items, int lambda, int32_t *ou,
                       int32_t *ov, float *ow, float aerr, float eps,
                       unsigned long long *stats) {
    using S = NpStage<NKS>;
    auto *fn = nearest_pairs_kernel<NKS, XR>;
    if (set_smem_attr(fn, S::SMEM, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NP_WARPS * 32, S::SMEM) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t want = (items + NP_WARPS - 1) / NP_WARPS;
    const int64_t cap = int64_t(ex.num_sms) * per_sm;
    const unsigned grid = unsigned(want < cap ? (want > 0 ? want : 1) : cap);
    FAMST_LAUNCH(ex, fn, grid, NP_WARPS * 32, S::SMEM, X, d, hr.h, hr.eb, hr.n2, members,
                 comp_off, item_off, out_off, t, items, lambda, ou, ov, ow, aerr, eps, stats);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace

size_t connect_nearest_workspace(int64_t n, int64_t t, int lambda) {
    // lists: sum over i of ceil(|C_i| / 32) (t - 1 - i) <= (n / 32 + t) t
    const int64_t lists = (n / 32 + t) * t;
    return 2 * align256(size_t(t + 1) * 8) + 3 * align256(size_t(lists) * lambda * 4) + 256;
}

// comp_off_host: the t + 1 member offsets on the host (the list layout is
// planned there). hr: BF16 rows of the points (ld <= 256).
famst_status connect_nearest(const Exec &ex, Arena &ar, const float *X, int d,
                             const HalfRows &hr, const int32_t *members,
                             const int32_t *comp_off, const int32_t *comp_off_host, int64_t t,
                             int lambda, int32_t *eu, int32_t *ev, float *ew, int32_t *eci,
                             int32_t *ecj, unsigned long long *stats) {
    if (t < 2) return FAMST_OK;
    if (!hr.h || hr.ld > 256) return FAMST_ERR_UNSUPPORTED;
    std::vector<int64_t> item_off(size_t(t + 1)), out_off(size_t(t + 1));
    item_off[0] = 0;
    out_off[0] = 0;
    for (int64_t i = 0; i < t; ++i) {
        const int64_t nb = (comp_off_host[i + 1] - comp_off_host[i] + 31) / 32;
        item_off[size_t(i + 1)] = item_off[size_t(i)] + nb;
        out_off[size_t(i + 1)] = out_off[size_t(i)] + nb * (t - 1 - i);
    }
    const int64_t items = item_off[size_t(t)], lists = out_off[size_t(t)];
    int64_t *d_item = ar.take<int64_t>(size_t(t + 1));
    int64_t *d_out = ar.take<int64_t>(size_t(t + 1));
    int32_t *ou = ar.take<int32_t>(size_t(lists) * lambda);
    int32_t *ov = ar.take<int32_t>(size_t(lists) * lambda);
    float *ow = ar.take<float>(size_t(lists) * lambda);
    if (!d_item || !d_out || !ou || !ov || !ow) return FAMST_ERR_OOM;
    if (cudaMemcpyAsync(d_item, item_off.data(), size_t(t + 1) * 8, cudaMemcpyHostToDevice,
                        ex.stream) != cudaSuccess ||
        cudaMemcpyAsync(d_out, out_off.data(), size_t(t + 1) * 8, cudaMemcpyHostToDevice,
                        ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    const float aerr = float(hr.ld * std::ldexp(1.0, -19) + std::ldexp(1.0, -20));
    const float eps = float((d + 16) * std::ldexp(1.0, -24) * 1.1);
    famst_status st;
    if (hr.ld == 64)
        st = launch_np<4, 2>(ex, X, d, hr, members, comp_off, d_item, d_out, t, items, lambda, ou,
                             ov, ow, aerr, eps, stats);
    else if (hr.ld == 128)
        st = launch_np<8, 4>(ex, X, d, hr, members, comp_off, d_item, d_out, t, items, lambda, ou,
                             ov, ow, aerr, eps, stats);
    else
        st = launch_np<16, 0>(ex, X, d, hr, members, comp_off, d_item, d_out, t, items, lambda,
                              ou, ov, ow, aerr, eps, stats);
    if (st != FAMST_OK) return st;
    // the host vectors must outlive the copies above
    if (cudaStreamSynchronize(ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    const int64_t npairs = t * (t - 1) / 2;
    int64_t mg = (npairs * 32 + 255) / 256;
    const int64_t mcap = int64_t(ex.num_sms) * 16;
    FAMST_LAUNCH(ex, nearest_merge_kernel, unsigned(mg < mcap ? mg : mcap), 256, 0, comp_off,
                 d_out, t, lambda, ou, ov, ow, eu, ev, ew, eci, ecj);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst
