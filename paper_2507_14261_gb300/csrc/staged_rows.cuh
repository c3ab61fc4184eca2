// Device pieces shared by the kernels that stage BF16 rows of the points in
// shared memory and take their dot products on the tensor cores
// (mma.sync m16n8k16): Algorithm 4's refinement scans and the
// nearest-pair variant of Algorithm 3. The rows are the centred BF16 copies
// h of the points with a per-row error bound eb >= ||h - (x - m)|| and norm
// ||h||^2 (HalfRows); every decision is taken on canonical FP32 distances,
// the BF16 dot products only rule candidates out with rigorous bounds.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "famst_internal.cuh"

namespace famst {
namespace staged {


// Staging buffer of one warp: 32 rows of LD BF16 values plus 16 bytes of
// padding, so the 8 rows an ldmatrix phase reads fall in 8 different
// 16-byte bank groups.
template <int NKS>
struct StageRows {
    static constexpr int LD = NKS * 16;         // row length (elements)
    static constexpr int RS = LD * 2 + 16;      // row stride in shared memory (bytes)
    static constexpr int ROWS_BYTES = 32 * RS;  // one round of 32 rows
};

// 16-byte global -> shared copy through the load/store unit, not cached in L1
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
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
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Copy the BF16 rows of the lanes' candidates (cand < 0: none) to the warp's
// buffer: CH 16-byte pieces per row, one instruction copying 32 / CH rows.
// Completes before returning.
template <int NKS>
__device__ __forceinline__ void stage_rows(const __nv_bfloat16 *__restrict__ H, int cand,
                                           uint32_t sbuf, int lane) {
    using S = StageRows<NKS>;
    constexpr int CH = S::LD * 2 / 16;
    constexpr int RPI = 32 / CH;
    const int ch = lane % CH, sub = lane / CH;
#pragma unroll
    for (int q = 0; q < CH; ++q) {
        const int slot = q * RPI + sub;
        const int cs = __shfl_sync(0xffffffffu, cand, slot);
        if (cs >= 0)
            cp_async16(sbuf + uint32_t(slot * S::RS + ch * 16), H + int64_t(cs) * S::LD + ch * 8);
    }
    cp_async_wait_all();
    __syncwarp();
}

// acc[T] = D of mma tile T: rows = candidates 16 T .. 16 T + 15 of the
// staged round, columns = the eight B columns (b0, b1 per k step).
template <int NKS>
__device__ __forceinline__ void round_dots(uint32_t sbuf, const uint32_t (&b0)[NKS],
                                           const uint32_t (&b1)[NKS], int lane,
                                           float (&acc)[2][4]) {
    using S = StageRows<NKS>;
    // ldmatrix: lanes 8 mi .. 8 mi + 7 address matrix mi = (rows 8 (mi & 1) ..,
    // k half mi >> 1): the A fragment order of m16n8k16
    const int mi = lane >> 3, rr = lane & 7;
    const uint32_t arow = sbuf + uint32_t(((mi & 1) * 8 + rr) * S::RS + (mi >> 1) * 16);
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
}

// Rigorous bounds [lo, hi] on the canonical distance from the BF16 dot
// product dt of centred rows with norms nx, ny and row error bounds ebx,
// eby: |p~ - ||h_x - h_y||^2| <= aerr (nx + ny) + 1e-35 with
// p~ = nx + ny - 2 dt, ||(h_y - h_x) - (y - x)|| <= ebx + eby, and eps for
// the canonical sum's own error; directed rounding throughout.
__device__ __forceinline__ void dist_bounds(float dt, float nx, float ny, float ebx, float eby,
                                            float aerr, float eps, float &lo, float &hi) {
    const float nn = __fadd_rn(nx, ny);
    const float pt = __fmaf_rn(-2.0f, dt, nn);
    const float A = __fmaf_ru(nn, aerr, 1e-35f);
    const float slo = __fsqrt_rd(fmaxf(__fsub_rd(pt, A), 0.0f));
    const float shi = __fsqrt_ru(__fadd_ru(pt, A));
    const float E = __fadd_ru(ebx, eby);
    lo = fmaxf(__fmul_rd(__fsub_rd(slo, E), 1.0f - eps), 0.0f);
    hi = __fmul_ru(__fadd_ru(shi, E), 1.0f + eps);
}

// Canonical FP32 distance of rows a and b by the whole warp (lane l holds
// partial l); XR > 0: d <= 32 XR, the rows are read as XR slices per lane.
template <int XR>
__device__ __forceinline__ float canon_w(const float *__restrict__ X, int d, int a, int b,
                                         int lane) {
    if constexpr (XR > 0) {
        float xa[XR], xb[XR];
#pragma unroll
        for (int q = 0; q < XR; ++q) {
            const int t = lane + 32 * q;
            xa[q] = t < d ? __ldg(X + int64_t(a) * d + t) : 0.0f;
            xb[q] = t < d ? __ldg(X + int64_t(b) * d + t) : 0.0f;
        }
        float p = 0.0f;
#pragma unroll
        for (int q = 0; q < XR; ++q) {
            const float dl = __fsub_rn(xb[q], xa[q]);
            p = __fmaf_rn(dl, dl, p);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
        return __fsqrt_rn(p);
    } else {
        return __fsqrt_rn(canon_p_warp(X + int64_t(a) * d, X + int64_t(b) * d, d, lane));
    }
}

__device__ __forceinline__ uint64_t cand_key(float w, int id) {
    return (uint64_t(__float_as_uint(w)) << 32) | uint32_t(id + 1);
}

}  // namespace staged
}  // namespace famst
