// Phase 2b (Algorithm 3) and Phase 3 (Algorithm 4) on the device.
//
// Connect: one warp per component pair (i < j). Lane l draws the samples
// s = l, l+32, ... of the pair with Philox4x32-10 (counter (s, p_lo, p_hi,
// 0), key = seed, p = i*t + j), maps the two 32-bit draws to members of
// C_i and C_j by multiply-shift, and computes the canonical distance of
// its samples. The lambda smallest (w, s) keys are then taken by lambda
// rounds of a warp-wide minimum, which yields them in ascending order --
// the "sort candidates, keep the first lambda" step of Algorithm 3.
//
// Refine: one warp per edge. A sweep of Algorithm 4 scans G[u] (kNN list
// of u plus its reverse edges) for the u' minimising w(u', v) and then
// G[v] against the new u (candidates first through a fast filter with
// rigorous bounds, the survivors decided on canonical distances). With the
// running best starting at the edge's
// own weight and a strict "<", the paper's ascending scan keeps the first
// (smallest id) of equal minima and keeps the incumbent on ties; that is
// an argmin under the key (w, 1 + id) with the incumbent keyed (w, 0), so
// lanes can scan in any order. Edges do not interact, so each warp
// repeats sweeps on its edge until it stops changing (bounded by
// max_iters); a histogram of per-edge change counts gives |Delta| of
// every global sweep.
#include <cuda_runtime.h>

#include <cmath>

#include "famst_internal.cuh"
#include "staged_rows.cuh"

namespace famst {
namespace {

__device__ __forceinline__ void pair_of(int64_t p, int64_t t, int64_t &i, int64_t &j) {
    // pairs enumerated i = 0.., j = i+1..t-1; start(i) = i*t - i*(i+1)/2
    double b = 2.0 * double(t) - 1.0;
    double disc = b * b - 8.0 * double(p);
    int64_t ii = int64_t((b - sqrt(disc > 0 ? disc : 0.0)) * 0.5);
    if (ii < 0) ii = 0;
    if (ii > t - 2) ii = t - 2;
    auto start = [t](int64_t x) { return x * t - x * (x + 1) / 2; };
    while (ii > 0 && start(ii) > p) --ii;
    while (ii + 1 <= t - 2 && start(ii + 1) <= p) ++ii;
    i = ii;
    j = p - start(ii) + ii + 1;
}

template <int PER, int VEC>
__global__ void connect_kernel(const float *__restrict__ X, int d,
                               const int32_t *__restrict__ members,
                               const int32_t *__restrict__ comp_off, int64_t t, int lambda,
                               uint64_t seed, int32_t *__restrict__ eu, int32_t *__restrict__ ev,
                               float *__restrict__ ew, int32_t *__restrict__ eci,
                               int32_t *__restrict__ ecj) {
    const int lane = threadIdx.x & 31;
    const int64_t npairs = t * (t - 1) / 2;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int L2 = lambda * lambda;
    const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
    for (int64_t pl = warp0; pl < npairs; pl += nwarps) {
        int64_t i, j;
        pair_of(pl, t, i, j);
        const uint64_t p = uint64_t(i) * uint64_t(t) + uint64_t(j);
        const int32_t oi = comp_off[i], oj = comp_off[j];
        const uint64_t si = uint64_t(comp_off[i + 1] - oi), sj = uint64_t(comp_off[j + 1] - oj);
        uint64_t kk[PER];
        int32_t uu[PER], vv[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            int s = lane + 32 * q;
            kk[q] = KEY_NONE;
            if (s < L2) {
                uint4 r = philox4x32_10(make_uint4(uint32_t(s), uint32_t(p), uint32_t(p >> 32), 0u),
                                        key);
                int32_t u = members[oi + int64_t((uint64_t(r.x) * si) >> 32)];
                int32_t v = members[oj + int64_t((uint64_t(r.y) * sj) >> 32)];
                float w = canon_dist<VEC>(X + int64_t(u) * d, X + int64_t(v) * d, d);
                kk[q] = nb_key(w, uint32_t(s));
                uu[q] = u;
                vv[q] = v;
            }
        }
        const int64_t ebase = pl * lambda;
        for (int r = 0; r < lambda; ++r) {
            uint64_t mine = KEY_NONE;
#pragma unroll
            for (int q = 0; q < PER; ++q) mine = kk[q] < mine ? kk[q] : mine;
            uint64_t best = warp_min_u64(mine);
            int s = int(key_lo(best));
            if ((s & 31) == lane) {
                int qq = s >> 5;
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    if (q == qq) {
                        kk[q] = KEY_NONE;
                        eu[ebase + r] = uu[q];
                        ev[ebase + r] = vv[q];
                        ew[ebase + r] = key_w(best);
                        eci[ebase + r] = int32_t(i);
                        ecj[ebase + r] = int32_t(j);
                    }
            }
        }
    }
}

// Filtered Algorithm 3 (rows 16-byte aligned, d % 4 == 0): the same draws,
// but the warp first computes fast squared distances of all lambda^2 pairs
// (grouped warp-wide sums, rows read contiguously) and evaluates the
// canonical distance (the whole warp, lane l holding partial l) only for
// pairs whose lower bound is within the lambda-th smallest upper bound
// (widened by 2^-20 for the rounding of sqrtf). At least lambda
// pairs have p_canon <= that bound, so every pair of the exact top lambda
// (w, s) survives, and the selection below sees the same winners.
template <int PER, int G>
__global__ void __launch_bounds__(256, 4) connect_filtered_kernel(const float *__restrict__ X, int d,
                                        const int32_t *__restrict__ members,
                                        const int32_t *__restrict__ comp_off, int64_t t,
                                        int lambda, uint64_t seed, float rho,
                                        int32_t *__restrict__ eu, int32_t *__restrict__ ev,
                                        float *__restrict__ ew, int32_t *__restrict__ eci,
                                        int32_t *__restrict__ ecj) {
    const int lane = threadIdx.x & 31;
    const int64_t npairs = t * (t - 1) / 2;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int L2 = lambda * lambda;
    const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
    const float widen = 1.0f + 0x1p-20f;
    __shared__ uint64_t s_kb[8][32 * PER];   // per warp: the draws' keys (hi, then w)
    __shared__ int32_t s_ub[8][32 * PER], s_vb[8][32 * PER];
    __shared__ float s_lob[8][32 * PER];
    const int wib = threadIdx.x >> 5;
    uint64_t *s_k = s_kb[wib];
    int32_t *s_u = s_ub[wib], *s_v = s_vb[wib];
    float *s_lo = s_lob[wib];
    for (int64_t pl = warp0; pl < npairs; pl += nwarps) {
        int64_t i, j;
        pair_of(pl, t, i, j);
        const uint64_t p = uint64_t(i) * uint64_t(t) + uint64_t(j);
        const int32_t oi = comp_off[i], oj = comp_off[j];
        const uint64_t si = uint64_t(comp_off[i + 1] - oi), sj = uint64_t(comp_off[j + 1] - oj);
        // one compiled copy of the draw body (unrolled copies stalled on
        // instruction fetch); a draw's state lives in its lane's slots of
        // shared memory (only that lane reads them back)
#pragma unroll 1
        for (int q = 0; q < PER; ++q) {
            const int s = lane + 32 * q;
            int32_t u = -1, v = -1;
            if (s < L2) {
                uint4 r = philox4x32_10(make_uint4(uint32_t(s), uint32_t(p), uint32_t(p >> 32), 0u),
                                        key);
                u = members[oi + int64_t((uint64_t(r.x) * si) >> 32)];
                v = members[oj + int64_t((uint64_t(r.y) * sj) >> 32)];
            }
            const float pf = warp_pairsq32g<G, 4>(X, d, u, v, lane);
            s_u[s] = u;
            s_v[s] = v;
            s_lo[s] = __fsub_rd(__fmul_rd(pf, 1.0f - rho), 1e-35f);
            s_k[s] = s < L2 ? nb_key(__fadd_ru(__fmul_ru(pf, 1.0f + rho), 1e-35f), uint32_t(s))
                            : KEY_NONE;
        }
        // the lambda-th smallest upper bound
        float H = 0.0f;
        {
            uint64_t hk[PER];
#pragma unroll
            for (int q = 0; q < PER; ++q) hk[q] = s_k[lane + 32 * q];
            for (int r = 0; r < lambda; ++r) {
                uint64_t mine = KEY_NONE;
#pragma unroll
                for (int q = 0; q < PER; ++q) mine = hk[q] < mine ? hk[q] : mine;
                const uint64_t best = warp_min_u64(mine);
                H = key_w(best);
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    if (hk[q] == best) hk[q] = KEY_NONE;
            }
        }
        const float bound = __fmul_ru(H, widen);
#pragma unroll 1
        for (int q = 0; q < PER; ++q) {
            const int s = lane + 32 * q;
            const int32_t u = s_u[s], v = s_v[s];
            uint64_t kq = KEY_NONE;
            // survivors: canonical distance by the whole warp, kept by their lane
            unsigned sv = __ballot_sync(0xffffffffu, s < L2 && s_lo[s] <= bound);
            while (sv) {
                const int sl = __ffs(sv) - 1;
                sv &= sv - 1;
                const int a = __shfl_sync(0xffffffffu, u, sl);
                const int b = __shfl_sync(0xffffffffu, v, sl);
                const float w = __fsqrt_rn(
                    canon_p_warp(X + int64_t(a) * d, X + int64_t(b) * d, d, lane));
                if (lane == sl) kq = nb_key(w, uint32_t(sl + 32 * q));
            }
            s_k[s] = kq;
        }
        uint64_t kk[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) kk[q] = s_k[lane + 32 * q];
        const int64_t ebase = pl * lambda;
        for (int r = 0; r < lambda; ++r) {
            uint64_t mine = KEY_NONE;
#pragma unroll
            for (int q = 0; q < PER; ++q) mine = kk[q] < mine ? kk[q] : mine;
            uint64_t best = warp_min_u64(mine);
            const int s = int(key_lo(best));
            if (best != KEY_NONE && (s & 31) == lane) {
                const int qq = s >> 5;
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    if (q == qq) kk[q] = KEY_NONE;
                eu[ebase + r] = s_u[s];
                ev[ebase + r] = s_v[s];
                ew[ebase + r] = key_w(best);
                eci[ebase + r] = int32_t(i);
                ecj[ebase + r] = int32_t(j);
            }
        }
    }
}

// 32 independent dot products of BF16 rows: lane l holds the pair (a[l],
// b[l]) (a < 0: none, result 0) and receives h_a . h_b. Groups of G = 8
// lanes read a row pair, lane g taking its 16-byte chunks g, g + 8, ...
// (V = ld / 64 of them); each lane sums its 8 V exact products by fmaf,
// then a transpose-sum inside the group (log2 G additions) gathers each
// pair's total: at most 8 V + 3 roundings, each within 2^-24 of the
// absolute sum of the products.
template <int V>
__device__ __forceinline__ float warp_pairdot32h(const __nv_bfloat16 *__restrict__ H, int ld,
                                                 int a, int b, int lane) {
    constexpr int G = 8, R = 32 / G;
    const int g = lane % G, h = lane / G;
    float acc[G];
#pragma unroll
    for (int s = 0; s < G; ++s) {
        const int ia = __shfl_sync(0xffffffffu, a, s * R + h);
        const int ib = __shfl_sync(0xffffffffu, b, s * R + h);
        const uint4 *ra = reinterpret_cast<const uint4 *>(H + int64_t(ia >= 0 ? ia : 0) * ld);
        const uint4 *rb = reinterpret_cast<const uint4 *>(H + int64_t(ia >= 0 ? ib : 0) * ld);
        float sum = 0.0f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint4 x = __ldg(ra + g + G * v), y = __ldg(rb + g + G * v);
            const uint32_t xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                sum = __fmaf_rn(__uint_as_float(xs[c] << 16), __uint_as_float(ys[c] << 16), sum);
                sum = __fmaf_rn(__uint_as_float(xs[c] & 0xffff0000u),
                                __uint_as_float(ys[c] & 0xffff0000u), sum);
            }
        }
        acc[s] = sum;
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

// Algorithm 3 with the filter on the centred BF16 rows of a build (half the
// bytes of the FP32 rows): the same draws; for every draw the bounds [lo, hi]
// on its canonical distance from the BF16 dot product, the rows' error
// bounds and norms (staged::dist_bounds); the canonical distance for the
// draws whose lo is within the lambda-th smallest hi, and the same selection
// by (w, sample index) as the other variants, so the edges are identical.
template <int PER, int V>
__global__ void __launch_bounds__(256, 4) connect_half_kernel(
    const float *__restrict__ X, int d, HalfRows hr, const int32_t *__restrict__ members,
    const int32_t *__restrict__ comp_off, int64_t t, int lambda, uint64_t seed, float aerr,
    float eps, int32_t *__restrict__ eu, int32_t *__restrict__ ev, float *__restrict__ ew,
    int32_t *__restrict__ eci, int32_t *__restrict__ ecj) {
    const int lane = threadIdx.x & 31;
    const int64_t npairs = t * (t - 1) / 2;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int L2 = lambda * lambda;
    const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
    const float widen = 1.0f + 0x1p-20f;
    __shared__ uint64_t s_kb[8][32 * PER];   // per warp: the draws' keys (hi, then w)
    __shared__ int32_t s_ub[8][32 * PER], s_vb[8][32 * PER];
    __shared__ float s_lob[8][32 * PER];
    const int wib = threadIdx.x >> 5;
    uint64_t *s_k = s_kb[wib];
    int32_t *s_u = s_ub[wib], *s_v = s_vb[wib];
    float *s_lo = s_lob[wib];
    for (int64_t pl = warp0; pl < npairs; pl += nwarps) {
        int64_t i, j;
        pair_of(pl, t, i, j);
        const uint64_t p = uint64_t(i) * uint64_t(t) + uint64_t(j);
        const int32_t oi = comp_off[i], oj = comp_off[j];
        const uint64_t si = uint64_t(comp_off[i + 1] - oi), sj = uint64_t(comp_off[j + 1] - oj);
        // one compiled copy of the draw body (unrolled copies stalled on
        // instruction fetch); a draw's state lives in its lane's slots of
        // shared memory (only that lane reads them back)
#pragma unroll 1
        for (int q = 0; q < PER; ++q) {
            const int s = lane + 32 * q;
            int32_t u = -1, v = -1;
            if (s < L2) {
                uint4 r = philox4x32_10(make_uint4(uint32_t(s), uint32_t(p), uint32_t(p >> 32), 0u),
                                        key);
                u = members[oi + int64_t((uint64_t(r.x) * si) >> 32)];
                v = members[oj + int64_t((uint64_t(r.y) * sj) >> 32)];
            }
            const float dt = warp_pairdot32h<V>(hr.h, hr.ld, u, v, lane);
            float l = __int_as_float(0x7f800000), h = 0.0f;
            if (s < L2)
                staged::dist_bounds(dt, __ldg(hr.n2 + u), __ldg(hr.n2 + v), __ldg(hr.eb + u),
                                    __ldg(hr.eb + v), aerr, eps, l, h);
            s_u[s] = u;
            s_v[s] = v;
            s_lo[s] = l;
            s_k[s] = s < L2 ? nb_key(h, uint32_t(s)) : KEY_NONE;
        }
        // the lambda-th smallest upper bound
        float H = 0.0f;
        {
            uint64_t hk[PER];
#pragma unroll
            for (int q = 0; q < PER; ++q) hk[q] = s_k[lane + 32 * q];
            for (int r = 0; r < lambda; ++r) {
                uint64_t mine = KEY_NONE;
#pragma unroll
                for (int q = 0; q < PER; ++q) mine = hk[q] < mine ? hk[q] : mine;
                const uint64_t best = warp_min_u64(mine);
                H = key_w(best);
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    if (hk[q] == best) hk[q] = KEY_NONE;
            }
        }
        const float bound = __fmul_ru(H, widen);
#pragma unroll 1
        for (int q = 0; q < PER; ++q) {
            const int s = lane + 32 * q;
            const int32_t u = s_u[s], v = s_v[s];
            uint64_t kq = KEY_NONE;
            // survivors: canonical distance by the whole warp, kept by their lane
            unsigned sv = __ballot_sync(0xffffffffu, s < L2 && s_lo[s] <= bound);
            while (sv) {
                const int sl = __ffs(sv) - 1;
                sv &= sv - 1;
                const int a = __shfl_sync(0xffffffffu, u, sl);
                const int b = __shfl_sync(0xffffffffu, v, sl);
                const float w = __fsqrt_rn(
                    canon_p_warp(X + int64_t(a) * d, X + int64_t(b) * d, d, lane));
                if (lane == sl) kq = nb_key(w, uint32_t(sl + 32 * q));
            }
            s_k[s] = kq;
        }
        uint64_t kk[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) kk[q] = s_k[lane + 32 * q];
        const int64_t ebase = pl * lambda;
        for (int r = 0; r < lambda; ++r) {
            uint64_t mine = KEY_NONE;
#pragma unroll
            for (int q = 0; q < PER; ++q) mine = kk[q] < mine ? kk[q] : mine;
            uint64_t best = warp_min_u64(mine);
            const int s = int(key_lo(best));
            if (best != KEY_NONE && (s & 31) == lane) {
                const int qq = s >> 5;
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    if (q == qq) kk[q] = KEY_NONE;
                eu[ebase + r] = s_u[s];
                ev[ebase + r] = s_v[s];
                ew[ebase + r] = key_w(best);
                eci[ebase + r] = int32_t(i);
                ecj[ebase + r] = int32_t(j);
            }
        }
    }
}

// Batched connect: pairs of every cloud in one index space. pp[b] (B+1,
// device) = number of pairs of clouds before b, cbase[b] (B+1) = the first
// global component index of cloud b; cloud b draws with key seed + b and the
// cloud-local pair index, exactly as a build of that cloud alone.
template <int PER, int VEC>
__global__ void connect_batched_kernel(const float *__restrict__ X, int ld, int dc,
                                       const int32_t *__restrict__ members,
                                       const int32_t *__restrict__ comp_off,
                                       const long long *__restrict__ pp,
                                       const int32_t *__restrict__ cbase, int B, int lambda,
                                       uint64_t seed, int64_t m_cap, int32_t *__restrict__ eu,
                                       int32_t *__restrict__ ev, float *__restrict__ ew,
                                       int32_t *__restrict__ eci, int32_t *__restrict__ ecj) {
    const int lane = threadIdx.x & 31;
    const int64_t npairs = pp[B];
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int L2 = lambda * lambda;
    for (int64_t pg = warp0; pg < npairs; pg += nwarps) {
        int lo = 0, hi = B;  // pp[lo] <= pg < pp[hi]
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (pp[mid] <= pg) lo = mid; else hi = mid;
        }
        const int b = lo;
        const int64_t t = cbase[b + 1] - cbase[b];
        const int64_t pl = pg - pp[b];
        int64_t i, j;
        pair_of(pl, t, i, j);
        const uint64_t p = uint64_t(i) * uint64_t(t) + uint64_t(j);
        const uint64_t sb = seed + uint64_t(b);
        const uint2 key = make_uint2(uint32_t(sb), uint32_t(sb >> 32));
        const int gi = cbase[b] + int(i), gj = cbase[b] + int(j);
        const int32_t oi = comp_off[gi], oj = comp_off[gj];
        const uint64_t si = uint64_t(comp_off[gi + 1] - oi), sj = uint64_t(comp_off[gj + 1] - oj);
        uint64_t kk[PER];
        int32_t uu[PER], vv[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            int s = lane + 32 * q;
            kk[q] = KEY_NONE;
            if (s < L2) {
                uint4 r = philox4x32_10(make_uint4(uint32_t(s), uint32_t(p), uint32_t(p >> 32), 0u),
                                        key);
                int32_t u = members[oi + int64_t((uint64_t(r.x) * si) >> 32)];
                int32_t v = members[oj + int64_t((uint64_t(r.y) * sj) >> 32)];
                float w = canon_dist<VEC>(X + int64_t(u) * ld, X + int64_t(v) * ld, dc);
                kk[q] = nb_key(w, uint32_t(s));
                uu[q] = u;
                vv[q] = v;
            }
        }
        const int64_t ebase = pg * lambda;
        for (int r = 0; r < lambda; ++r) {
            uint64_t mine = KEY_NONE;
#pragma unroll
            for (int q = 0; q < PER; ++q) mine = kk[q] < mine ? kk[q] : mine;
            uint64_t best = warp_min_u64(mine);
            int s = int(key_lo(best));
            if ((s & 31) == lane && ebase + r < m_cap) {
                int qq = s >> 5;
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    if (q == qq) {
                        kk[q] = KEY_NONE;
                        eu[ebase + r] = uu[q];
                        ev[ebase + r] = vv[q];
                        ew[ebase + r] = key_w(best);
                        eci[ebase + r] = gi;
                        ecj[ebase + r] = gj;
                    }
            } else if ((s & 31) == lane) {
                int qq = s >> 5;
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    if (q == qq) kk[q] = KEY_NONE;
            }
        }
    }
}

// argmin over the adjacency of `c` (kNN list + reverse edges) of the
// candidate key (w(cand, fixed), 1 + cand); incumbent keyed (w0, 0).
// Direct version: each lane streams its candidate's row from global memory.
template <int VEC>
__device__ __forceinline__ uint64_t scan_side(const float *__restrict__ X, int d, int c,
                                              int fixed, int other, int want_comp, float w0,
                                              const int32_t *__restrict__ nbr, int k,
                                              const int32_t *__restrict__ rev_off,
                                              const int32_t *__restrict__ rev_src,
                                              const int32_t *__restrict__ comp, int lane,
                                              unsigned &evals) {
    uint64_t best = uint64_t(__float_as_uint(w0)) << 32;
    const int r0 = rev_off[c], r1 = rev_off[c + 1];
    const int deg = k + (r1 - r0);
    const float *xf = X + int64_t(fixed) * d;
    for (int idx = lane; idx < deg; idx += 32) {
        int cand = idx < k ? nbr[int64_t(c) * k + idx] : rev_src[r0 + idx - k];
        if (comp[cand] != want_comp || cand == other) continue;  // G[c] ∩ C, and u' != v
        ++evals;
        float w = canon_dist<VEC>(X + int64_t(cand) * d, xf, d);
        uint64_t key = (uint64_t(__float_as_uint(w)) << 32) | uint32_t(cand + 1);
        best = key < best ? key : best;
    }
    return warp_min_u64(best);
}

// Filtered version (rows 16-byte aligned, d % 4 == 0, d <= 512): the warp
// first computes fast squared distances of its 32 candidates with the
// grouped warp-wide sums (every row read contiguously by G lanes), then
// evaluates canonical distances (the whole warp per candidate, lane l
// holding partial l) only for candidates the fast value cannot rule out.
// The fast and the canonical sums add the same rounded terms
// fl(x_t - y_t)^2 in different orders, so both lie within gamma_n of the
// exact sum: p_canon / p_fast is within [1 - rho, 1 + rho]. A candidate
// whose lower bound exceeds (a) the smallest upper bound in the round or
// (b) the current best weight squared, both widened by 2^-20 for the
// rounding of sqrtf, cannot be the argmin under (w, id); the others are
// decided on canonical weights, so the result equals scan_side's.
template <int G>
__device__ __forceinline__ uint64_t scan_side_filtered(
    const float *__restrict__ X, int d, int c, int fixed, int other, int want_comp, float w0,
    const int32_t *__restrict__ nbr, int k, const int32_t *__restrict__ rev_off,
    const int32_t *__restrict__ rev_src, const int32_t *__restrict__ comp, int lane, float rho,
    unsigned &evals, unsigned &canon, bool check) {
    const float *xf = X + int64_t(fixed) * d;
    float4 fx[4];
    row_slices_g<G, 4>(xf, d >> 2, lane, fx);
    uint64_t best = uint64_t(__float_as_uint(w0)) << 32;
    const int r0 = rev_off[c], r1 = rev_off[c + 1];
    const int deg = k + (r1 - r0);
    const float widen = 1.0f + 0x1p-20f;
    const float inf = __int_as_float(0x7f800000);
    for (int base = 0; base < deg; base += 32) {
        const int idx = base + lane;
        int cand = -1;
        if (idx < deg) {
            cand = idx < k ? nbr[int64_t(c) * k + idx] : rev_src[r0 + idx - k];
            // G[c] ∩ C and u' != v (checked for caller-supplied labels)
            if (check && (comp[cand] != want_comp || cand == other)) cand = -1;
        }
        const unsigned live = __ballot_sync(0xffffffffu, cand >= 0);
        if (live == 0u) continue;
        if (lane == 0) evals += unsigned(__popc(live));
        float lo = inf, hi = inf;
        const float pf = warp_sqdist32g<G, 4>(X, d, fx, fixed, cand, lane);
        if (cand >= 0) {
            lo = __fsub_rd(__fmul_rd(pf, 1.0f - rho), 1e-35f);
            hi = __fadd_ru(__fmul_ru(pf, 1.0f + rho), 1e-35f);
        }
        float mh = hi;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) mh = fminf(mh, __shfl_xor_sync(0xffffffffu, mh, o));
        const float wb = key_w(best);
        const float bound = fminf(__fmul_ru(mh, widen), __fmul_ru(__fmul_ru(wb, wb), widen));
        // survivors are decided on canonical distances, each by the whole warp
        unsigned sv = __ballot_sync(0xffffffffu, cand >= 0 && lo <= bound);
        if (lane == 0) canon += unsigned(__popc(sv));
        while (sv) {
            const int sl = __ffs(sv) - 1;
            sv &= sv - 1;
            const int c2 = __shfl_sync(0xffffffffu, cand, sl);
            const float w = __fsqrt_rn(canon_p_warp(X + int64_t(c2) * d, xf, d, lane));
            const uint64_t key = (uint64_t(__float_as_uint(w)) << 32) | uint32_t(c2 + 1);
            best = key < best ? key : best;   // the same in every lane
        }
    }
    return best;
}

// Process edges in the order `order` (component-pair tiles, so the rows in
// flight stay in L2), each to its own fixed point.
// Four resident blocks per SM (64 registers): the scans are latency bound,
// and occupancy buys more than the few spilled registers cost.
template <int VEC, int G>
__global__ void __launch_bounds__(256, 4) refine_kernel(const float *__restrict__ X, int d,
                              const int32_t *__restrict__ nbr, int k,
                              const int32_t *__restrict__ rev_off,
                              const int32_t *__restrict__ rev_src,
                              const int32_t *__restrict__ comp, int32_t *__restrict__ eu,
                              int32_t *__restrict__ ev, float *__restrict__ ew,
                              const int32_t *__restrict__ eci, const int32_t *__restrict__ ecj,
                              const int32_t *__restrict__ order, int64_t m,
                              const int64_t *__restrict__ m_dev, int max_iters,
                              int32_t *__restrict__ change_hist,
                              unsigned long long *__restrict__ next_item, int *dstatus,
                              float rho, unsigned long long *__restrict__ evals_out, bool check) {
    if (m_dev) m = *m_dev < m ? *m_dev : m;  // device-side edge count, capped by capacity
    const int lane = threadIdx.x & 31;
    unsigned long long evals_total = 0, canon_total = 0;   // evaluations of this lane
    // Edges are handed out one at a time from a global counter, so the
    // edges in flight stay a narrow window of `order` (and their rows in L2)
    // even though edges need different numbers of sweeps.
    while (true) {
        unsigned long long w0 = 0;
        if (lane == 0) w0 = atomicAdd(next_item, 1ull);
        const int64_t w = int64_t(__shfl_sync(0xffffffffu, w0, 0));
        if (w >= m) break;
        const int64_t e = order ? int64_t(order[w]) : w;
        int u = eu[e], v = ev[e];
        float wt = ew[e];
        const int ci = eci[e], cj = ecj[e];
        int changes = 0;
        unsigned evals = 0, canon = 0;
        // The v-scan is a function of (v, u*) alone (C_i and C_j are disjoint,
        // so the exclusion of u never bites, and its incumbent is w(u*, v)).
        // When a sweep leaves v in place and the next one leaves u in place,
        // the second v-scan repeats the first: its result is reused.
        int mv_v = -1, mv_u = -1;
        uint64_t mv_b = 0;
        for (; changes < max_iters; ++changes) {
            uint64_t bu, bv;
            int us, vs;
            float ws;
            // u-loop: u' in G[u] ∩ C_i, u' != v, against v
            if constexpr (G > 0)
                bu = scan_side_filtered<G>(X, d, u, v, v, ci, wt, nbr, k, rev_off, rev_src, comp,
                                           lane, rho, evals, canon, check);
            else
                bu = scan_side<VEC>(X, d, u, v, v, ci, wt, nbr, k, rev_off, rev_src, comp, lane,
                                    evals);
            us = key_lo(bu) ? int(key_lo(bu)) - 1 : u;
            ws = key_w(bu);
            // v-loop: v' in G[v] ∩ C_j, v' != u, against the new u*
            if (v == mv_v && us == mv_u)
                bv = mv_b;
            else if constexpr (G > 0)
                bv = scan_side_filtered<G>(X, d, v, us, u, cj, ws, nbr, k, rev_off, rev_src, comp,
                                           lane, rho, evals, canon, check);
            else
                bv = scan_side<VEC>(X, d, v, us, u, cj, ws, nbr, k, rev_off, rev_src, comp, lane,
                                    evals);
            mv_v = v;
            mv_u = us;
            mv_b = bv;
            vs = key_lo(bv) ? int(key_lo(bv)) - 1 : v;
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
        canon_total += G > 0 ? canon : evals;
    }
    if (evals_out) {   // [0] candidate distances, [1] canonical evaluations among them
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            evals_total += __shfl_xor_sync(0xffffffffu, evals_total, o);
            canon_total += __shfl_xor_sync(0xffffffffu, canon_total, o);
        }
        if (lane == 0) {
            atomicAdd(evals_out, evals_total);
            atomicAdd(evals_out + 1, canon_total);
        }
    }
}

// Launch of the refinement kernel in the variant the shape allows: the FP32
// grouped filter for 16-byte rows with 32 <= d <= 512, else the canonical
// distance per lane. (Builds with BF16 rows use refine_build, which stages
// rows in shared memory.) Persistent grid; edges are fetched from
// *next_item (zeroed by the caller).
famst_status launch_refine(const Exec &ex, const float *X, int d, bool vec4, const int32_t *nbr,
                           int k, const int32_t *rev_off, const int32_t *rev_src,
                           const int32_t *comp, int32_t *eu, int32_t *ev, float *ew,
                           const int32_t *eci, const int32_t *ecj, const int32_t *order,
                           int64_t m, const int64_t *m_dev, int max_iters, int32_t *change_hist,
                           unsigned long long *next_item, unsigned long long *evals, bool check,
                           int *variant) {
    const int th = 256;
    const int G = (vec4 && d >= 32) ? sq_group(d) : 0;
    const void *fn = G == 2 ? (const void *)refine_kernel<4, 2>
                   : G == 4 ? (const void *)refine_kernel<4, 4>
                   : G == 8 ? (const void *)refine_kernel<4, 8>
                   : G == 16 ? (const void *)refine_kernel<4, 16>
                   : G == 32 ? (const void *)refine_kernel<4, 32>
                   : vec4 ? (const void *)refine_kernel<4, 0>
                          : (const void *)refine_kernel<1, 0>;
    // persistent grid: as many blocks as stay resident
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, th, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t want = (m * 32 + th - 1) / th;
    int64_t cap = int64_t(ex.num_sms) * per_sm;
    unsigned grid = unsigned(want < cap ? want : cap);
    if (grid == 0) grid = 1;
    const float rho = fast_rho(d, 1);
    if (variant) *variant = G > 0 ? REFINE_FILTER_FP32 : REFINE_FILTER_NONE;
#define REFINE_LAUNCH(V, GG)                                                                     \
    FAMST_LAUNCH(ex, (refine_kernel<V, GG>), grid, th, 0, X, d, nbr, k, rev_off, rev_src, comp, \
                 eu, ev, ew, eci, ecj, order, m, m_dev, max_iters, change_hist, next_item,       \
                 ex.dstatus, rho, evals, check)
    timer_mark(ex, TIMER_REFINE, false);
    switch (G) {
        case 2: REFINE_LAUNCH(4, 2); break;
        case 4: REFINE_LAUNCH(4, 4); break;
        case 8: REFINE_LAUNCH(4, 8); break;
        case 16: REFINE_LAUNCH(4, 16); break;
        case 32: REFINE_LAUNCH(4, 32); break;
        default:
            if (vec4) REFINE_LAUNCH(4, 0);
            else REFINE_LAUNCH(1, 0);
    }
    timer_mark(ex, TIMER_REFINE, true);
#undef REFINE_LAUNCH
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

// Centre m for the BF16 rows: the mean of up to 256 evenly spaced rows (any
// m is valid; the bounds use the actual fl(x - m)).
__global__ void half_mean_kernel(const float *__restrict__ X, int64_t n, int d,
                                 float *__restrict__ m) {
    const int64_t S = n < 256 ? n : 256;
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
        float s = 0.0f;
        int64_t i = 0;
        for (; i + 8 <= S; i += 8) {   // eight independent loads in flight
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __ldg(X + ((i + q) * n / S) * d + t);
#pragma unroll
            for (int q = 0; q < 8; ++q) s += v[q];
        }
        for (; i < S; ++i) s += __ldg(X + (i * n / S) * d + t);
        m[t] = s / float(S);
    }
}

// h = bf16(fl(x - m)), zero beyond d; eb >= ||h - (x - m)||: the BF16
// rounding error of this row itself, ||h - fl(x - m)|| (each difference
// exact, squares summed rounding up), plus the centring rounding (each
// coordinate within 2^-24 of x - m), with margins for the square roots and
// a tiny absolute term for BF16 subnormals. One warp per row; n2 = ||h||^2.
__global__ void half_rows_kernel(const float *__restrict__ X, int64_t n, int d, int ld,
                                 const float *__restrict__ m, __nv_bfloat16 *__restrict__ h,
                                 float *__restrict__ eb, float *__restrict__ n2) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    float acc = 0.0f, acch = 0.0f, accr = 0.0f;
    for (int t = lane; t < ld; t += 32) {
        const float x = t < d ? __fsub_rn(__ldg(X + r * d + t), __ldg(m + t)) : 0.0f;
        const __nv_bfloat16 hb = __float2bfloat16_rn(x);
        h[r * ld + t] = hb;
        acc = __fmaf_ru(x, x, acc);
        const float hf = __bfloat162float(hb);
        acch = __fmaf_rn(hf, hf, acch);
        const float e = __fsub_rn(hf, x);   // exact: hf is x rounded to 8 bits
        accr = __fmaf_ru(e, e, accr);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        acc = __fadd_ru(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        acch = __fadd_rn(acch, __shfl_xor_sync(0xffffffffu, acch, o));
        accr = __fadd_ru(accr, __shfl_xor_sync(0xffffffffu, accr, o));
    }
    if (lane == 0) {
        const float nrm = __fmul_ru(__fsqrt_ru(acc), 1.0f + 0x1p-12f);
        const float rnd = __fmul_ru(__fsqrt_ru(accr), 1.0f + 0x1p-12f);
        eb[r] = __fadd_ru(__fadd_ru(rnd, __fmul_ru(nrm, 0x1p-22f)), 1e-30f);
        n2[r] = acch;   // within ld 2^-23 of ||h||^2
    }
}

// tile key of an edge: its component pair's (ci / TT, cj / TT) cell
__global__ void edge_tile_key_kernel(const int32_t *__restrict__ eci,
                                     const int32_t *__restrict__ ecj, int64_t m, int tt, int T,
                                     uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    keys[e] = uint32_t(eci[e] / tt) * uint32_t(T) + uint32_t(ecj[e] / tt);
    vals[e] = int32_t(e);
}

}  // namespace

famst_status connect_edges(const Exec &ex, const float *X, int d, bool vec4,
                           const int32_t *members, const int32_t *comp_off, int64_t t,
                           int lambda, uint64_t seed, int32_t *eu, int32_t *ev, float *ew,
                           int32_t *eci, int32_t *ecj, const HalfRows *hr) {
    if (t < 2) return FAMST_OK;
    int64_t npairs = t * (t - 1) / 2;
    int per = (lambda * lambda + 31) / 32;
    // BF16 rows of a build (ld = 64 .. 256): the filter reads those
    if (hr && hr->h && hr->ld >= 64 && hr->ld <= 256 && per <= 4) {
        const int th = 256;
        const int64_t want = (npairs * 32 + th - 1) / th;
        const int64_t cap = int64_t(ex.num_sms) * 16;
        const unsigned grid = unsigned(want < cap ? want : cap);
        // |p~ - ||h_a - h_b||^2| <= aerr (||h_a||^2 + ||h_b||^2): each norm
        // within ld 2^-23 of its value, the dot within (8 V + 3) 2^-24 of the
        // products' absolute sum (<= the half sum of the norms), the final
        // rounding of p~; taken with a factor-two margin. eps: the canonical
        // sum's own error, as for the refinement.
        const float aerr = float(hr->ld * std::ldexp(1.0, -22) + std::ldexp(1.0, -18));
        const float eps = float((d + 16) * std::ldexp(1.0, -24) * 1.1);
        const int V = hr->ld / 64;
#define CONNECT_H(P, VV)                                                                        \
    FAMST_LAUNCH(ex, (connect_half_kernel<P, VV>), grid, th, 0, X, d, *hr, members, comp_off, t, \
                 lambda, seed, aerr, eps, eu, ev, ew, eci, ecj)
#define CONNECT_HV(P)                                                                          \
    do {                                                                                       \
        if (V == 1) CONNECT_H(P, 1);                                                           \
        else if (V == 2) CONNECT_H(P, 2);                                                      \
        else if (V == 3) CONNECT_H(P, 3);                                                      \
        else CONNECT_H(P, 4);                                                                  \
    } while (0)
        timer_mark(ex, TIMER_CONNECT, false);
        if (per <= 1) CONNECT_HV(1);
        else if (per <= 2) CONNECT_HV(2);
        else CONNECT_HV(4);
        timer_mark(ex, TIMER_CONNECT, true);
#undef CONNECT_HV
#undef CONNECT_H
        return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
    }
    // filtered variant for the common shapes (lambda <= 11, 32 <= d <= 256)
    const int Gs = (vec4 && d >= 32) ? sq_group(d) : 0;
    const int G = (per <= 4 && (Gs == 4 || Gs == 8 || Gs == 16)) ? Gs : 0;
    const int th = 256;
    int64_t want = (npairs * 32 + th - 1) / th;
    int64_t cap = int64_t(ex.num_sms) * 16;
    unsigned grid = unsigned(want < cap ? want : cap);
    const float rho = fast_rho(d, 1);
#define CONNECT_F(P, GG)                                                                      \
    FAMST_LAUNCH(ex, (connect_filtered_kernel<P, GG>), grid, th, 0, X, d, members, comp_off, t, \
                 lambda, seed, rho, eu, ev, ew, eci, ecj)
    if (G > 0) {
        timer_mark(ex, TIMER_CONNECT, false);
        if (per <= 1) {
            if (G == 4) CONNECT_F(1, 4); else if (G == 8) CONNECT_F(1, 8); else CONNECT_F(1, 16);
        } else if (per <= 2) {
            if (G == 4) CONNECT_F(2, 4); else if (G == 8) CONNECT_F(2, 8); else CONNECT_F(2, 16);
        } else {
            if (G == 4) CONNECT_F(4, 4); else if (G == 8) CONNECT_F(4, 8); else CONNECT_F(4, 16);
        }
        timer_mark(ex, TIMER_CONNECT, true);
        return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
    }
#define CONNECT_CASE(P)                                                                       \
    if (per <= P) {                                                                           \
        if (vec4)                                                                             \
            FAMST_LAUNCH(ex, (connect_kernel<P, 4>), grid, th, 0, X, d, members, comp_off, t,  \
                         lambda, seed, eu, ev, ew, eci, ecj);                                 \
        else                                                                                  \
            FAMST_LAUNCH(ex, (connect_kernel<P, 1>), grid, th, 0, X, d, members, comp_off, t,  \
                         lambda, seed, eu, ev, ew, eci, ecj);                                 \
        return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;                 \
    }
    CONNECT_CASE(1)
    CONNECT_CASE(2)
    CONNECT_CASE(4)
    CONNECT_CASE(8)
    CONNECT_CASE(16)
    CONNECT_CASE(32)
#undef CONNECT_CASE
#undef CONNECT_F
    return FAMST_ERR_UNSUPPORTED;
}

size_t half_rows_workspace(int64_t n, int d) {
    const int ld = (d + 63) / 64 * 64;
    return align256(size_t(n) * ld * 2) + align256(size_t(n) * 4) * 2 + align256(size_t(d) * 4);
}

famst_status half_rows(const Exec &ex, Arena &ar, const float *X, int64_t n, int d,
                       HalfRows *out) {
    const int ld = (d + 63) / 64 * 64;
    __nv_bfloat16 *h = ar.take<__nv_bfloat16>(size_t(n) * ld);
    float *eb = ar.take<float>(size_t(n));
    float *n2 = ar.take<float>(size_t(n));
    float *m = ar.take<float>(size_t(d));
    if (!h || !eb || !n2 || !m) return FAMST_ERR_OOM;
    FAMST_LAUNCH(ex, half_mean_kernel, 1, 256, 0, X, n, d, m);
    FAMST_LAUNCH(ex, half_rows_kernel, unsigned((n * 32 + 255) / 256), 256, 0, X, n, d, ld, m, h,
                 eb, n2);
    out->h = h;
    out->ld = ld;
    out->eb = eb;
    out->m = m;
    out->n2 = n2;
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

size_t refine_workspace(int64_t m) {
    return align256(size_t(m) * 4) * 2 + 256 + radix_sort_workspace(m);
}

famst_status refine_edges(const Exec &ex, Arena &ar, const float *X, int d, bool vec4,
                          const int32_t *nbr, int k, const int32_t *rev_off,
                          const int32_t *rev_src, const int32_t *comp, int64_t t, int32_t *eu,
                          int32_t *ev, float *ew, const int32_t *eci, const int32_t *ecj,
                          int64_t m, int max_iters, int32_t *change_hist,
                          unsigned long long *evals, bool check, int *variant) {
    if (m == 0) return FAMST_OK;
    // order: stable sort of the edges by component-pair tile
    constexpr int TT = 24;
    const int T = int((t + TT - 1) / TT);
    uint32_t *keys = ar.take<uint32_t>(size_t(m));
    int32_t *order = ar.take<int32_t>(size_t(m));
    unsigned long long *next_item = ar.take<unsigned long long>(1);
    if (!keys || !order || !next_item) return FAMST_ERR_OOM;
    if (cudaMemsetAsync(next_item, 0, 8, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, edge_tile_key_kernel, unsigned((m + 255) / 256), 256, 0, eci, ecj, m, TT, T,
                 keys, order);
    int bits = 0;
    while ((int64_t(1) << bits) < int64_t(T) * T) ++bits;
    famst_status st = radix_sort_pairs(ex, ar, keys, order, m, bits);
    if (st != FAMST_OK) return st;
    return launch_refine(ex, X, d, vec4, nbr, k, rev_off, rev_src, comp, eu, ev, ew, eci, ecj, order,
                         m, nullptr, max_iters, change_hist, next_item, evals, check, variant);
}

}  // namespace famst

namespace famst {

// Refinement of E with a device-side edge count (at most m_cap), edges in
// their stored order; nothing here synchronises with the host.
famst_status refine_edges_dev(const Exec &ex, Arena &ar, const float *X, int d, bool vec4,
                              const int32_t *nbr, int k, const int32_t *rev_off,
                              const int32_t *rev_src, const int32_t *comp, int32_t *eu,
                              int32_t *ev, float *ew, const int32_t *eci, const int32_t *ecj,
                              int64_t m_cap, const int64_t *m_dev, int max_iters,
                              int32_t *change_hist) {
    if (m_cap == 0) return FAMST_OK;
    unsigned long long *next_item = ar.take<unsigned long long>(1);
    if (!next_item) return FAMST_ERR_OOM;
    if (cudaMemsetAsync(next_item, 0, 8, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    return launch_refine(ex, X, d, vec4, nbr, k, rev_off, rev_src, comp, eu, ev, ew, eci, ecj,
                         nullptr, m_cap, m_dev, max_iters, change_hist, next_item, nullptr,
                         false, nullptr);
}

}  // namespace famst

namespace famst {

famst_status connect_edges_batched(const Exec &ex, const float *X, int ld, int dc,
                                   const int32_t *members, const int32_t *comp_off,
                                   const long long *pp, const int32_t *cbase, int B, int lambda,
                                   uint64_t seed, int64_t m_cap, int32_t *eu, int32_t *ev,
                                   float *ew, int32_t *eci, int32_t *ecj) {
    int per = (lambda * lambda + 31) / 32;
    const int th = 256;
    unsigned grid = unsigned(ex.num_sms) * 16;
#define CONNECT_B_CASE(P)                                                                          \
    if (per <= P) {                                                                                \
        FAMST_LAUNCH(ex, (connect_batched_kernel<P, 4>), grid, th, 0, X, ld, dc, members, comp_off, \
                     pp, cbase, B, lambda, seed, m_cap, eu, ev, ew, eci, ecj);                     \
        return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;                   \
    }
    CONNECT_B_CASE(1)
    CONNECT_B_CASE(2)
    CONNECT_B_CASE(4)
    CONNECT_B_CASE(8)
    CONNECT_B_CASE(16)
    CONNECT_B_CASE(32)
#undef CONNECT_B_CASE
    return FAMST_ERR_UNSUPPORTED;
}

}  // namespace famst
