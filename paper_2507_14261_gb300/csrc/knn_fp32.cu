// Phase 1 (Algorithm 1, GetANNs) as exact brute force on FP32 SIMT tiles.
//
// A block owns QM = 64 query rows and sweeps key tiles of KN = 128 points.
// For every (query, key) pair the block computes the canonical distance
// chain p = fmaf(x_t - y_t, x_t - y_t, p) over t = 0..d-1 in order, so the
// p values are bit-identical to the oracle's and need no re-rank. Dims are
// staged through shared memory in chunks of DC = 32 (transposed, double
// buffered); each thread accumulates a 4 x 8 register micro-tile.
//
// Selection is fused: the tile of p values goes to shared memory, then
// SPR threads per query row each scan a strided slice of the tile's
// columns against the slice's current k-th key and insert into a private
// sorted list of (w, id) keys. Only rows that beat the running threshold
// cost more than one compare, so the n x n matrix never leaves the SM.
// At the end of a block's key range the SPR slice lists of each row are
// merged. When the key range is split over S blocks (small n), partial
// lists go to global memory and a merge kernel finishes them.
#include <cuda_runtime.h>

#include "famst_internal.cuh"

namespace famst {
namespace {

constexpr int QM = 64;
constexpr int KN = 128;
constexpr int DC = 32;
constexpr int NT = 256;
constexpr int KS_STRIDE = KN + 4;   // floats per dim row of the key stage
constexpr int PS_STRIDE = KN + 1;   // floats per query row of the p tile

__host__ __device__ inline int spr_for(int k) { return k <= 32 ? 4 : (k <= 64 ? 2 : 1); }

struct KnnSmem {
    static size_t bytes(int k) {
        size_t stage = size_t(DC) * QM + size_t(DC) * KS_STRIDE;  // floats
        size_t ps = size_t(QM) * PS_STRIDE;
        size_t lists = size_t(k) * QM * spr_for(k);  // uint64
        return (2 * stage + ps) * sizeof(float) + lists * sizeof(uint64_t) +
               size_t(QM) * 4 * sizeof(int);  // list counts
    }
};

__global__ void __launch_bounds__(NT, 1)
knn_fp32_kernel(const float *__restrict__ X, int n, int d, int ld, int k,
                const int32_t *__restrict__ qrows, int64_t q0, int nq,
                int tiles_per_split, uint64_t *__restrict__ part,
                int32_t *__restrict__ nbr, float *__restrict__ dist,
                const F32Tile *__restrict__ btab, const int32_t *__restrict__ colcomp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int spr = spr_for(k);
    const int nsel = QM * spr;
    float *stage = reinterpret_cast<float *>(smem_raw);
    const int stage_floats = DC * QM + DC * KS_STRIDE;
    float *Ps = stage + 2 * stage_floats;
    uint64_t *L = reinterpret_cast<uint64_t *>(Ps + QM * PS_STRIDE);
    int *Lcnt = reinterpret_cast<int *>(L + size_t(k) * nsel);

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    int qbase = blockIdx.x * QM;
    const int split = blockIdx.y;
    int tile_begin, tile_end, shift = 0, key_base = 0;
    if (btab) {
        // batched: one block per 64 query rows of one cloud, keys = the cloud
        const F32Tile T = btab[blockIdx.x];
        tile_begin = T.tile0;
        tile_end = T.tile1;
        key_base = T.key_base;
        n = T.key_end;
        d = T.d;
        shift = T.shift;
        nq = T.nq;
        q0 = T.qbase;
        qbase = 0;
    } else {
        const int ntiles_total = (n + KN - 1) / KN;
        tile_begin = split * tiles_per_split;
        tile_end = min(ntiles_total, tile_begin + tiles_per_split);
    }
    const int nchunks = (d + DC - 1) / DC;

    // query ids of this block's rows (for the self test and the loads)
    __shared__ int qid_s[QM];
    if (tid < QM) {
        int q = qbase + tid;
        qid_s[tid] = q < nq ? (qrows ? qrows[q] : int(q0 + q)) : -1;
    }
    // selection state
    const bool selector = tid < nsel;
    const int srow = tid / spr, sslice = tid % spr;
    int lcount = 0;
    uint64_t kth = KEY_NONE;
    float pthr = __int_as_float(0x7f800000);
    __syncthreads();
    const int my_qid = selector ? qid_s[srow] : -1;
    // optional component mask: keys in the query's own component are skipped
    const int my_comp = (colcomp && my_qid >= 0) ? colcomp[my_qid] : -1;

    // register prefetch of one chunk: 16 key floats + 8 query floats
    float kreg[16], qreg[8];
    auto load_chunk = [&](int tile, int c) {
        int key0 = key_base + tile * KN;
        int t0 = c * DC;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            int idx = tid + NT * r;
            int j = idx >> 5, t = idx & 31;
            int row = key0 + j, col = t0 + t;
            kreg[r] = (row < n && col < d) ? __ldg(X + int64_t(row) * ld + col) : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int idx = tid + NT * r;
            int i = idx >> 5, t = idx & 31;
            int qi = qid_s[i], col = t0 + t;
            qreg[r] = (qi >= 0 && col < d) ? __ldg(X + int64_t(qi) * ld + col) : 0.0f;
        }
    };
    auto store_chunk = [&](int buf) {
        float *Qs = stage + buf * stage_floats;
        float *Ks = Qs + DC * QM;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            int idx = tid + NT * r;
            Ks[(idx & 31) * KS_STRIDE + (idx >> 5)] = kreg[r];
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int idx = tid + NT * r;
            Qs[(idx & 31) * QM + (idx >> 5)] = qreg[r];
        }
    };

    int buf = 0;
    if (tile_begin < tile_end) load_chunk(tile_begin, 0);
    for (int tile = tile_begin; tile < tile_end; ++tile) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

        for (int c = 0; c < nchunks; ++c) {
            store_chunk(buf);
            __syncthreads();
            // prefetch the next chunk (or the next tile's first chunk)
            if (c + 1 < nchunks) load_chunk(tile, c + 1);
            else if (tile + 1 < tile_end) load_chunk(tile + 1, 0);
            const float *Qs = stage + buf * stage_floats;
            const float *Ks = Qs + DC * QM;
#pragma unroll 8
            for (int t = 0; t < DC; ++t) {
                float4 a = *reinterpret_cast<const float4 *>(Qs + t * QM + ty * 4);
                float4 b0 = *reinterpret_cast<const float4 *>(Ks + t * KS_STRIDE + tx * 4);
                float4 b1 = *reinterpret_cast<const float4 *>(Ks + t * KS_STRIDE + 64 + tx * 4);
                float av[4] = {a.x, a.y, a.z, a.w};
                float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float dl = __fsub_rn(av[i], bv[j]);
                        acc[i][j] = __fmaf_rn(dl, dl, acc[i][j]);
                    }
            }
            buf ^= 1;
        }
        // p tile to shared memory
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float *prow = Ps + (ty * 4 + i) * PS_STRIDE;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                prow[tx * 4 + j] = acc[i][j];
                prow[64 + tx * 4 + j] = acc[i][4 + j];
            }
        }
        __syncthreads();
        if (selector && my_qid >= 0) {
            const int key0 = key_base + tile * KN;
            const float *prow = Ps + srow * PS_STRIDE;
            uint64_t *Lme = L + tid;
            for (int cidx = sslice; cidx < KN; cidx += spr) {
                int j = key0 + cidx;
                float p = prow[cidx];
                if (!(p <= pthr) || j >= n || j == my_qid) continue;
                if (colcomp && colcomp[j] == my_comp) continue;
                uint64_t key = nb_key(__fsqrt_rn(p), uint32_t(j));
                if (key >= kth) continue;
                int pos = lcount < k ? lcount++ : k - 1;
                while (pos > 0) {
                    uint64_t prev = Lme[size_t(pos - 1) * nsel];
                    if (prev <= key) break;
                    Lme[size_t(pos) * nsel] = prev;
                    --pos;
                }
                Lme[size_t(pos) * nsel] = key;
                if (lcount == k) {
                    kth = Lme[size_t(k - 1) * nsel];
                    float wk = key_w(kth);
                    pthr = wk * wk * (1.0f + 0x1p-20f);
                }
            }
        }
        // Ps is rewritten only after the next tile's first chunk barrier
    }

    // merge the spr slice lists of each row
    if (selector) Lcnt[tid] = lcount;
    __syncthreads();
    if (tid < QM && qbase + tid < nq) {
        const int r = tid;
        int head[4] = {0, 0, 0, 0};
        int cnt[4] = {0, 0, 0, 0};
        for (int s = 0; s < spr; ++s) cnt[s] = Lcnt[r * spr + s];
        const int64_t q = qbase + r;
        for (int o = 0; o < k; ++o) {
            uint64_t best = KEY_NONE;
            int bs = -1;
            for (int s = 0; s < spr; ++s) {
                if (head[s] < cnt[s]) {
                    uint64_t v = L[size_t(head[s]) * nsel + r * spr + s];
                    if (v < best) { best = v; bs = s; }
                }
            }
            if (bs >= 0) head[bs]++;
            if (part) {
                part[(size_t(split) * nq + q) * k + o] = best;
            } else {
                const int64_t orow = btab ? int64_t(q0 + q - shift) : (qrows ? int64_t(qrows[q]) : q);
                nbr[orow * k + o] = best == KEY_NONE ? -1 : int32_t(key_lo(best)) - shift;
                dist[orow * k + o] = best == KEY_NONE ? __int_as_float(0x7f800000) : key_w(best);
            }
        }
    }
}

// S sorted partial lists per row -> the k smallest keys.
__global__ void knn_merge_kernel(const uint64_t *__restrict__ part, int S, int nq, int k,
                                 const int32_t *__restrict__ qrows, int32_t *__restrict__ nbr,
                                 float *__restrict__ dist) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    int head[64];
    for (int s = 0; s < S; ++s) head[s] = 0;
    for (int o = 0; o < k; ++o) {
        uint64_t best = KEY_NONE;
        int bs = -1;
        for (int s = 0; s < S; ++s) {
            if (head[s] < k) {
                uint64_t v = part[(size_t(s) * nq + q) * k + head[s]];
                if (v < best) { best = v; bs = s; }
            }
        }
        if (bs >= 0) head[bs]++;
        const int64_t orow = qrows ? int64_t(qrows[q]) : int64_t(q);
        nbr[orow * k + o] = best == KEY_NONE ? -1 : int32_t(key_lo(best));
        dist[orow * k + o] = best == KEY_NONE ? __int_as_float(0x7f800000) : key_w(best);
    }
}

struct SplitPlan {
    int qblocks, S, tiles_per_split;
};

SplitPlan plan(int64_t n, int64_t nq, int num_sms) {
    SplitPlan p;
    p.qblocks = int((nq + QM - 1) / QM);
    int ntiles = int((n + KN - 1) / KN);
    int want = (2 * num_sms + p.qblocks - 1) / p.qblocks;
    int S = want < 1 ? 1 : (want > 64 ? 64 : want);
    if (S > ntiles) S = ntiles;
    p.tiles_per_split = (ntiles + S - 1) / S;
    p.S = (ntiles + p.tiles_per_split - 1) / p.tiles_per_split;
    return p;
}

}  // namespace

size_t knn_fp32_workspace(int64_t n, int d, int k, int64_t nq, int num_sms) {
    (void)d;
    SplitPlan p = plan(n, nq, num_sms);
    if (p.S <= 1) return 0;
    return align256(size_t(p.S) * nq * k * sizeof(uint64_t));
}

famst_status knn_fp32(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, int k,
                      const int32_t *qrows, int64_t q0, int64_t nq, int32_t *nbr, float *dist,
                      const int32_t *colcomp) {
    if (nq == 0) return FAMST_OK;
    if (k < 1 || k > 128) return FAMST_ERR_UNSUPPORTED;
    SplitPlan p = plan(n, nq, ex.num_sms);
    size_t smem = KnnSmem::bytes(k);
    if (set_smem_attr(knn_fp32_kernel, int(smem), ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    uint64_t *part = nullptr;
    if (p.S > 1) {
        part = ar.take<uint64_t>(size_t(p.S) * nq * k);
        if (!part) return FAMST_ERR_OOM;
    }
    dim3 grid(p.qblocks, p.S);
    FAMST_LAUNCH(ex, knn_fp32_kernel, grid, NT, smem, X, int(n), d, d, k, qrows, q0, int(nq),
                 p.tiles_per_split, part, nbr, dist, nullptr, colcomp);
    if (cudaPeekAtLastError() != cudaSuccess) return FAMST_ERR_CUDA;
    if (p.S > 1) {
        int th = 128;
        FAMST_LAUNCH(ex, knn_merge_kernel, int((nq + th - 1) / th), th, 0, part, p.S, int(nq),
                     k, qrows, nbr, dist);
        if (cudaPeekAtLastError() != cudaSuccess) return FAMST_ERR_CUDA;
    }
    return FAMST_OK;
}

}  // namespace famst

namespace famst {

// Batched exact kNN on FP32 tiles: one block per entry of `tiles` (64 query
// rows of one cloud against that cloud's keys), X in the padded row space
// with row stride ld; ids are written in the compact space.
famst_status knn_fp32_batched(const Exec &ex, const float *Xp, int ld, int k, const F32Tile *tiles,
                              int64_t nblocks, int32_t *nbr, float *dist) {
    if (nblocks == 0) return FAMST_OK;
    if (k < 1 || k > 128) return FAMST_ERR_UNSUPPORTED;
    size_t smem = KnnSmem::bytes(k);
    if (set_smem_attr(knn_fp32_kernel, int(smem), ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, knn_fp32_kernel, dim3(unsigned(nblocks), 1), NT, smem, Xp, 0, 0, ld, k,
                 nullptr, 0, 0, 0, nullptr, nbr, dist, tiles, nullptr);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst
