// Phase 1 (Algorithm 1, GetANNs) as exact brute force on FP32 SIMT tiles.
//
// A block owns QM = 64 query rows and sweeps key tiles of KN = 128 points.
// For every (query, key) pair the block computes a fast squared distance
// p = sum of fmaf(x_t - y_t, x_t - y_t, .) over t = 0..d-1 in order (dims
// staged through shared memory in chunks of DC = 32, transposed, double
// buffered; each thread accumulates a 4 x 8 register micro-tile). It keeps
// the k' = k + 8 best (sqrt p, id) of every row; the canonical re-rank below
// computes their canonical distances, sorts them, and certifies the row when
// the FP32 error bound proves no unkept point can reach the k-th canonical
// distance. Rows it cannot certify (ties at the boundary) are recomputed by
// an exact warp-per-row brute force on canonical distances.
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
                const int64_t orow = btab ? int64_t(q0 + q - shift) : q;
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
        nbr[int64_t(q) * k + o] = best == KEY_NONE ? -1 : int32_t(key_lo(best));
        dist[int64_t(q) * k + o] = best == KEY_NONE ? __int_as_float(0x7f800000) : key_w(best);
    }
}

// ------------------------------------------------------------ exactness

constexpr int FP32_MARGIN = 8;   // candidates kept beyond k for the certificate

// Bitonic sort of 128 keys held 4 per lane (element h * 32 + lane), ascending.
__device__ __forceinline__ void warp_sort128(uint64_t (&key)[4], int lane) {
#pragma unroll
    for (int size = 2; size <= 128; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int hs = stride >> 5;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    if (h & hs) continue;
                    const int e = h * 32 + lane;
                    const bool asc = (e & size) == 0;
                    const uint64_t a = key[h], b = key[h | hs];
                    const uint64_t mn = a < b ? a : b, mx = a < b ? b : a;
                    key[h] = asc ? mn : mx;
                    key[h | hs] = asc ? mx : mn;
                }
            } else {
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int e = h * 32 + lane;
                    const bool asc = (e & size) == 0;
                    const uint64_t other = shfl_xor_u64(key[h], stride);
                    const bool lower = (lane & stride) == 0;
                    const uint64_t mn = key[h] < other ? key[h] : other;
                    const uint64_t mx = key[h] < other ? other : key[h];
                    key[h] = (lower == asc) ? mn : mx;
                }
            }
        }
    }
}

// Canonical re-rank of the FP32 tiles' kp candidates, one warp per query
// row q (point i = qrows[q] or q0 + q): canonical distances, sort by (w, id),
// certificate. Every unkept point has fast distance >= the kp-th kept one's,
// sp; fast and canonical sums of the same rounded terms differ by a factor
// within 1 +- rho, so an unkept point's canonical distance is at least
// sp (1 - rho) and the row is certified when that exceeds the k-th.
template <int VEC>
__global__ void rerank_fp32_kernel(const float *__restrict__ X, int d, int k, int kp,
                                   int64_t nq, const int32_t *__restrict__ qrows, int64_t q0,
                                   const int32_t *__restrict__ cand, const float *__restrict__ wf,
                                   float rho, int32_t *__restrict__ nbr, float *__restrict__ dist,
                                   int32_t *__restrict__ fail_rows,
                                   int32_t *__restrict__ fail_count) {
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const int64_t i = qrows ? int64_t(qrows[q]) : q0 + q;
    const float *xi = X + i * d;
    uint64_t key[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int p = h * 32 + lane;
        key[h] = KEY_NONE;
        if (p < kp) {
            const int j = cand[q * kp + p];
            if (j >= 0) key[h] = nb_key(canon_dist<VEC>(xi, X + int64_t(j) * d, d), uint32_t(j));
        }
    }
    warp_sort128(key, lane);
    const uint64_t kth = shfl_idx_u64(key[(k - 1) >> 5], (k - 1) & 31);
    const int jl = cand[q * kp + kp - 1];
    const float sp = jl >= 0 ? wf[q * kp + kp - 1] : __int_as_float(0x7f800000);
    const bool cert = !(sp < __int_as_float(0x7f800000)) ||
                      (kth != KEY_NONE && double(sp) * (1.0 - double(rho)) > double(key_w(kth)));
    if (cert) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int e = h * 32 + lane;
            if (e < k) {
                nbr[i * k + e] = key[h] == KEY_NONE ? -1 : int32_t(key_lo(key[h]));
                dist[i * k + e] = key[h] == KEY_NONE ? __int_as_float(0x7f800000) : key_w(key[h]);
            }
        }
    } else if (lane == 0) {
        fail_rows[atomicAdd(fail_count, 1)] = int32_t(i);
    }
}

// Canonical squared distances of 32 keys (lane l's key `cand`, < 0: none)
// to one point whose coordinates t = l + 32 j lane l holds in xs[j]: lane l
// accumulates partial l of every key (coalesced loads), a butterfly
// transpose-sum then leaves key l's canonical value in lane l -- at every
// stage a lane adds the same pair of partial sums the canonical butterfly
// adds, for the key whose result it keeps.
template <int DJ>
__device__ __forceinline__ float warp_canon32(const float *__restrict__ X, int d,
                                              const float (&xs)[DJ], int self, int cand,
                                              int lane) {
    float acc[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        const int id = __shfl_sync(0xffffffffu, cand, s);
        const float *row = X + int64_t(id >= 0 ? id : self) * d;
        float a = 0.0f;
#pragma unroll
        for (int j = 0; j < DJ; ++j) {
            const int t = lane + 32 * j;
            if (t < d) {
                const float x = __fsub_rn(__ldg(row + t), xs[j]);
                a = __fmaf_rn(x, x, a);
            }
        }
        acc[s] = a;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? acc[i] : acc[i + o];
            const float keep = up ? acc[i + o] : acc[i];
            acc[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
    }
    return cand >= 0 ? acc[0] : 0.0f;
}

// Insert key K into the warp's sorted list L (element h * 32 + lane, KEY_NONE
// at the end); the last element drops out.
__device__ __forceinline__ void warp_list_insert(uint64_t (&L)[4], uint64_t K, int lane) {
    int pos = 0;
#pragma unroll
    for (int h = 0; h < 4; ++h) pos += __popc(__ballot_sync(0xffffffffu, L[h] < K));
    uint64_t prev[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const uint64_t up = shfl_up_u64(L[h], 1);
        const uint64_t wrap = h > 0 ? shfl_idx_u64(L[h > 0 ? h - 1 : 0], 31) : KEY_NONE;
        prev[h] = lane == 0 ? wrap : up;
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int e = h * 32 + lane;
        L[h] = e < pos ? L[h] : (e == pos ? K : prev[h]);
    }
}

// Exact kNN of single rows on canonical distances, one warp per row of
// rows[0 .. *count): keys in rounds of 32 (warp_canon32), the k best (w, id)
// in a warp-wide sorted list. colcomp: keys of the row's own component are
// skipped. k <= 128; d <= 32 DJ, or DJ = 0 for any d.
template <int DJ>
__global__ void exact_rows_kernel(const float *__restrict__ X, int64_t n, int d, int k,
                                  const int32_t *__restrict__ rows,
                                  const int32_t *__restrict__ count,
                                  const int32_t *__restrict__ colcomp, int32_t *__restrict__ nbr,
                                  float *__restrict__ dist) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int nrows = *count;
    for (int64_t q = w0; q < nrows; q += nw) {
        const int i = rows[q];
        float xs[DJ > 0 ? DJ : 1];
#pragma unroll
        for (int j = 0; j < DJ; ++j) {
            const int t = lane + 32 * j;
            xs[j] = t < d ? __ldg(X + int64_t(i) * d + t) : 0.0f;
        }
        const int my_comp = colcomp ? colcomp[i] : -1;
        uint64_t L[4] = {KEY_NONE, KEY_NONE, KEY_NONE, KEY_NONE};
        uint64_t kth = KEY_NONE;
        for (int64_t base = 0; base < n; base += 32) {
            const int64_t j = base + lane;
            int cand = (j < n && j != i) ? int(j) : -1;
            if (cand >= 0 && colcomp && colcomp[cand] == my_comp) cand = -1;
            if (__ballot_sync(0xffffffffu, cand >= 0) == 0u) continue;
            float p;
            if constexpr (DJ > 0) {
                p = warp_canon32<DJ>(X, d, xs, i, cand, lane);
            } else {   // any d: one key at a time, the whole warp per key
                p = 0.0f;
                for (int s = 0; s < 32; ++s) {
                    const int id = __shfl_sync(0xffffffffu, cand, s);
                    const float ps = canon_p_warp(X + int64_t(i) * d,
                                                  X + int64_t(id >= 0 ? id : i) * d, d, lane);
                    if (lane == s) p = ps;
                }
            }
            const uint64_t key = cand >= 0 ? nb_key(__fsqrt_rn(p), uint32_t(cand)) : KEY_NONE;
            unsigned pass = __ballot_sync(0xffffffffu, key < kth);
            while (pass) {
                const int s = __ffs(pass) - 1;
                pass &= pass - 1;
                const uint64_t K = shfl_idx_u64(key, s);
                if (K < kth) {
                    warp_list_insert(L, K, lane);
                    kth = shfl_idx_u64(L[(k - 1) >> 5], (k - 1) & 31);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int e = h * 32 + lane;
            if (e < k) {
                nbr[int64_t(i) * k + e] = L[h] == KEY_NONE ? -1 : int32_t(key_lo(L[h]));
                dist[int64_t(i) * k + e] = L[h] == KEY_NONE ? __int_as_float(0x7f800000) : key_w(L[h]);
            }
        }
    }
}

__device__ __forceinline__ int cloud_index(const long long *__restrict__ off, int B, long long v) {
    int lo = 0, hi = B;  // off[lo] <= v < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

// Batched canonical re-rank: one block per FP32 tile, a warp per row; rows,
// ids and the distance rows live in the compact space Xc (row stride ld,
// zero beyond each cloud's d). The same certificate as rerank_fp32_kernel.
__global__ void rerank_fp32_batched_kernel(const float *__restrict__ Xc, int ld,
                                           const long long *__restrict__ voff, int B,
                                           const CloudDev *__restrict__ cl, int k, int kp,
                                           const F32Tile *__restrict__ tiles,
                                           const int32_t *__restrict__ cand,
                                           const float *__restrict__ wf, int32_t *__restrict__ nbr,
                                           float *__restrict__ dist, int32_t *__restrict__ fails,
                                           int32_t *__restrict__ nfail) {
    const F32Tile T = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int q = wib; q < T.nq; q += blockDim.x >> 5) {
        const int64_t v = int64_t(T.qbase) + q;
        const CloudDev c = cl[cloud_index(voff, B, v)];
        const int dc = (c.d + 3) & ~3;
        const double u = 1.0 / 16777216.0, nu = double(dc + 9) * u;
        const double rho = 2.01 * nu / (1.0 - nu) + 4.0 * u;
        const float *xi = Xc + v * ld;
        uint64_t key[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int p = h * 32 + lane;
            key[h] = KEY_NONE;
            if (p < kp) {
                const int j = cand[v * kp + p];
                if (j >= 0) key[h] = nb_key(canon_dist<4>(xi, Xc + int64_t(j) * ld, dc), uint32_t(j));
            }
        }
        warp_sort128(key, lane);
        const uint64_t kth = shfl_idx_u64(key[(k - 1) >> 5], (k - 1) & 31);
        const int jl = cand[v * kp + kp - 1];
        const float sp = jl >= 0 ? wf[v * kp + kp - 1] : __int_as_float(0x7f800000);
        const bool cert = !(sp < __int_as_float(0x7f800000)) ||
                          (kth != KEY_NONE && double(sp) * (1.0 - rho) > double(key_w(kth)));
        if (cert) {
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int e = h * 32 + lane;
                if (e < k) {
                    nbr[v * k + e] = key[h] == KEY_NONE ? -1 : int32_t(key_lo(key[h]));
                    dist[v * k + e] = key[h] == KEY_NONE ? __int_as_float(0x7f800000) : key_w(key[h]);
                }
            }
        } else if (lane == 0) {
            fails[atomicAdd(nfail, 1)] = int32_t(v);
        }
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

int fp32_kp(int64_t n, int k) {
    int64_t kp = k + FP32_MARGIN;
    if (kp > n - 1) kp = n - 1;
    if (kp > 128) kp = 128;
    return int(kp < k ? k : kp);
}

size_t knn_fp32_workspace(int64_t n, int d, int k, int64_t nq, int num_sms) {
    (void)d;
    const int kp = fp32_kp(n, k);
    SplitPlan p = plan(n, nq, num_sms);
    size_t b = align256(size_t(nq) * kp * 4) * 2 + align256(size_t(nq) * 4) + 256;
    if (p.S > 1) b += align256(size_t(p.S) * nq * kp * sizeof(uint64_t));
    return b;
}

// The FP32 tiles alone: the k best (sqrt p_fast, id) of every query row,
// rows written in query order q (not at qrows[q]).
famst_status knn_fp32_fast(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, int k,
                           const int32_t *qrows, int64_t q0, int64_t nq, int32_t *nbr,
                           float *dist, const int32_t *colcomp) {
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

famst_status exact_rows(const Exec &ex, const float *X, int64_t n, int d, int k,
                        const int32_t *rows, const int32_t *count, int64_t max_rows,
                        const int32_t *colcomp, int32_t *nbr, float *dist) {
    if (max_rows == 0) return FAMST_OK;
    if (k < 1 || k > 128) return FAMST_ERR_UNSUPPORTED;
    int64_t warps = max_rows < int64_t(ex.num_sms) * 16 ? max_rows : int64_t(ex.num_sms) * 16;
    const unsigned grid = unsigned((warps * 32 + 127) / 128);
    const int dj = (d + 31) / 32;
#define EXACT(DJV)                                                                              \
    FAMST_LAUNCH(ex, exact_rows_kernel<DJV>, grid, 128, 0, X, n, d, k, rows, count, colcomp, nbr, \
                 dist)
    if (dj <= 1) EXACT(1);
    else if (dj <= 2) EXACT(2);
    else if (dj <= 4) EXACT(4);
    else if (dj <= 8) EXACT(8);
    else if (dj <= 16) EXACT(16);
    else EXACT(0);
#undef EXACT
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

famst_status knn_fp32(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, int k,
                      const int32_t *qrows, int64_t q0, int64_t nq, int32_t *nbr, float *dist,
                      const int32_t *colcomp) {
    if (nq == 0) return FAMST_OK;
    if (k < 1 || k > 128 || k > n - 1) return FAMST_ERR_UNSUPPORTED;
    const int kp = fp32_kp(n, k);
    int32_t *cn = ar.take<int32_t>(size_t(nq) * kp);
    float *wf = ar.take<float>(size_t(nq) * kp);
    int32_t *fails = ar.take<int32_t>(size_t(nq));
    int32_t *nfail = ar.take<int32_t>(1);
    if (!cn || !wf || !fails || !nfail) return FAMST_ERR_OOM;
    famst_status st = knn_fp32_fast(ex, ar, X, n, d, kp, qrows, q0, nq, cn, wf, colcomp);
    if (st != FAMST_OK) return st;
    if (cudaMemsetAsync(nfail, 0, 4, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    const float rho = fast_rho(d, 1);
    const unsigned rgrid = unsigned((nq * 32 + 255) / 256);
    if ((d & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0)
        FAMST_LAUNCH(ex, rerank_fp32_kernel<4>, rgrid, 256, 0, X, d, k, kp, nq, qrows, q0, cn, wf,
                     rho, nbr, dist, fails, nfail);
    else
        FAMST_LAUNCH(ex, rerank_fp32_kernel<1>, rgrid, 256, 0, X, d, k, kp, nq, qrows, q0, cn, wf,
                     rho, nbr, dist, fails, nfail);
    if (cudaPeekAtLastError() != cudaSuccess) return FAMST_ERR_CUDA;
    return exact_rows(ex, X, n, d, k, fails, nfail, nq, colcomp, nbr, dist);
}

}  // namespace famst

namespace famst {

// Batched exact kNN on FP32 tiles: one block per entry of `tiles` (64 query
// rows of one cloud against that cloud's keys) keeps kp candidates per row,
// then the batched canonical re-rank, then exact rows for the uncertified.
famst_status knn_fp32_batched(const Exec &ex, const float *Xc, int ld, const long long *voff,
                              int B, const CloudDev *cl, int k, int kp, const F32Tile *tiles,
                              int64_t nblocks, int32_t *c, float *w, int32_t *fails,
                              int32_t *nfail, int32_t *nbr, float *dist) {
    if (nblocks == 0) return FAMST_OK;
    if (k < 1 || k > 64 || kp < k || kp > 128) return FAMST_ERR_UNSUPPORTED;
    size_t smem = KnnSmem::bytes(kp);
    if (set_smem_attr(knn_fp32_kernel, int(smem), ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, knn_fp32_kernel, dim3(unsigned(nblocks), 1), NT, smem, Xc, 0, 0, ld, kp,
                 nullptr, 0, 0, 0, nullptr, c, w, tiles, nullptr);
    if (cudaMemsetAsync(nfail, 0, 4, ex.stream) != cudaSuccess) return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, rerank_fp32_batched_kernel, unsigned(nblocks), 256, 0, Xc, ld, voff, B, cl, k,
                 kp, tiles, c, w, nbr, dist, fails, nfail);
    if (cudaPeekAtLastError() != cudaSuccess) return FAMST_ERR_CUDA;
    return fallback_rows_batched(ex, Xc, ld, voff, B, cl, k, fails, nfail, nbr, dist);
}

}  // namespace famst
