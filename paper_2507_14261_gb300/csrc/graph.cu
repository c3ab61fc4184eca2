// Phase 2a (Algorithm 2) on the device, plus the integer building blocks
// the later phases share: exclusive scan, stable LSD radix sort, and the
// reverse adjacency of the kNN graph.
//
// Algorithm 2 finds the components of the undirected graph G (every kNN
// edge taken both ways) by depth-first search from vertices 0, 1, 2, ...
// The search discovers each component at its smallest vertex id, so the
// component index it assigns equals the rank of that smallest id. The
// device computes the same partition with lock-free union-find (hook the
// larger root under the smaller with atomicCAS, path splitting in find),
// which also leaves the smallest id as each root; ranking the roots gives
// the discovery order.
#include <cuda_runtime.h>

#include "famst_internal.cuh"

namespace famst {
namespace {

constexpr int SCAN_NT = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

__device__ __forceinline__ int warp_incl_scan(int v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ int block_excl_scan(int v, int &excl) {
    __shared__ int wsum[33];  // 32 warp offsets + the block total
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? wsum[lane] : 0;
        int si = warp_incl_scan(s);
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wsum[32] = si;
    }
    __syncthreads();
    excl = inc - v + wsum[w];
    int total = wsum[32];
    __syncthreads();
    return total;
}

__global__ void scan_reduce_kernel(const int32_t *__restrict__ in, int64_t count,
                                   int32_t *__restrict__ bsum) {
    int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
    int s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        int64_t i = base + r * SCAN_NT + threadIdx.x;
        if (i < count) s += in[i];
    }
    int excl;
    int total = block_excl_scan(s, excl);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// single block: exclusive scan of the block sums in place; total to *total
__global__ void scan_blocksums_kernel(int32_t *__restrict__ bsum, int64_t nb,
                                      int32_t *__restrict__ total) {
    int carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int excl;
        int t = block_excl_scan(v, excl);
        if (i < nb) bsum[i] = carry + excl;
        carry += t;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_apply_kernel(const int32_t *__restrict__ in, int32_t *__restrict__ out,
                                  int64_t count, const int32_t *__restrict__ bsum) {
    // blocked per-thread ranges keep the sequential order inside a tile
    int64_t base = int64_t(blockIdx.x) * SCAN_TILE + int64_t(threadIdx.x) * SCAN_IPT;
    int v[SCAN_IPT];
    int s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        int64_t i = base + r;
        v[r] = i < count ? in[i] : 0;
        s += v[r];
    }
    int excl;
    block_excl_scan(s, excl);
    int run = bsum[blockIdx.x] + excl;
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        int64_t i = base + r;
        if (i < count) out[i] = run;
        run += v[r];
    }
}

// ------------------------------------------------------------ radix sort

constexpr int RS_NT = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_NT * RS_ROUNDS;

__global__ void rs_hist_kernel(const uint32_t *__restrict__ keys, int64_t count, int shift,
                               int32_t *__restrict__ hist, int nblocks) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = int64_t(blockIdx.x) * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + r * RS_NT + threadIdx.x;
        if (i < count) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[int64_t(threadIdx.x) * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter_kernel(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                  uint32_t *__restrict__ kout, int32_t *__restrict__ vout,
                                  int64_t count, int shift, const int32_t *__restrict__ offs,
                                  int nblocks) {
    __shared__ int basepos[256];
    __shared__ int wcnt[RS_NT / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    basepos[threadIdx.x] = offs[int64_t(threadIdx.x) * nblocks + blockIdx.x];
    for (int q = 0; q < RS_NT / 32; ++q) wcnt[q][threadIdx.x] = 0;
    __syncthreads();
    int64_t base = int64_t(blockIdx.x) * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + r * RS_NT + threadIdx.x;
        bool valid = i < count;
        uint32_t key = valid ? kin[i] : 0u;
        int32_t val = valid ? vin[i] : 0;
        int digit = valid ? int((key >> shift) & 255) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int lrank = __popc(peers & ((1u << lane) - 1u));
        bool leader = lrank == 0;
        if (leader && valid) wcnt[w][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pre = 0;
            for (int q = 0; q < w; ++q) pre += wcnt[q][digit];
            int pos = basepos[digit] + pre + lrank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int tot = 0;
        for (int q = 0; q < RS_NT / 32; ++q) {
            tot += wcnt[q][threadIdx.x];
            wcnt[q][threadIdx.x] = 0;
        }
        basepos[threadIdx.x] += tot;
        __syncthreads();
    }
}

// ----------------------------------------------------------- union-find

constexpr int UF_LIMIT = 1 << 22;

// Root of v. Path splitting; parent[x] <= x always holds. Volatile: other
// threads hook and compress concurrently, every read must see memory. At
// most `limit` steps: a find cut short raises STATUS_LOOP_LIMIT (the call
// then fails with FAMST_ERR_TIMEOUT) and returns an ancestor of v.
__device__ __forceinline__ int uf_find(int32_t *parent_, int v, int limit, int *dstatus) {
    volatile int32_t *parent = parent_;
    int p = parent[v];
    int guard = 0;
    while (p != v && guard++ < limit) {
        int g = parent[p];
        if (g != p) parent[v] = g;  // benign race: any ancestor is valid
        v = p;
        p = g;
    }
    if (p != v) set_status(dstatus, STATUS_LOOP_LIMIT);
    return v;
}

__global__ void uf_init_kernel(int32_t *parent, int64_t n) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) parent[v] = int32_t(v);
}

// Vertices in a scrambled order: thread e takes edge j = e mod k of vertex
// v = (e / k) * 0x9E3779B1 mod 2^m (odd multiplier: a bijection of
// [0, 2^m), 2^m >= n; v >= n idle). When ids are contiguous in space (clouds
// laid out one after another, sorted inputs), threads in flight together
// would otherwise all hook onto the same few roots.
__global__ void uf_hook_kernel(const int32_t *__restrict__ nbr, int64_t n, int k,
                               uint32_t vmask, int32_t *parent, int limit, int *dstatus) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t vl = e / k;
    if (vl > int64_t(vmask)) return;
    const uint32_t v = (uint32_t(vl) * 0x9E3779B1u) & vmask;
    if (int64_t(v) >= n) return;
    int a = int(v), b = nbr[int64_t(v) * k + (e - vl * k)];
    int ra = uf_find(parent, a, limit, dstatus), rb = uf_find(parent, b, limit, dstatus);
    for (int it = 0; it < limit; ++it) {
        if (ra == rb) return;
        int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
        int old = atomicCAS(&parent[hi], hi, lo);
        if (old == hi) return;
        // hi was hooked meanwhile: continue from its new parent
        if (ra > rb) ra = uf_find(parent, old, limit, dstatus);
        else rb = uf_find(parent, old, limit, dstatus);
    }
    set_status(dstatus, STATUS_LOOP_LIMIT);
}

// Roots go to a separate array: a concurrent find may still rewrite
// parent[v] with a non-root ancestor after this thread stored the root.
__global__ void uf_flatten_kernel(int32_t *parent, int64_t n, int32_t *root,
                                  int32_t *is_root, int limit, int *dstatus) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int r = uf_find(parent, int(v), limit, dstatus);
    root[v] = r;
    is_root[v] = (r == v) ? 1 : 0;
}

__global__ void uf_label_kernel(const int32_t *__restrict__ root, const int32_t *__restrict__ rank,
                                int64_t n, int32_t *__restrict__ comp) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = rank[root[v]];
}

__global__ void iota_keys_kernel(const int32_t *__restrict__ comp, int64_t n,
                                 uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) {
        keys[v] = uint32_t(comp[v]);
        vals[v] = int32_t(v);
    }
}

__global__ void segment_starts_kernel(const uint32_t *__restrict__ keys, int64_t n, int64_t t,
                                      int32_t *__restrict__ off) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n && (i == 0 || keys[i] != keys[i - 1])) off[keys[i]] = int32_t(i);
    if (i == 0) off[t] = int32_t(n);
}

__global__ void count_in_kernel(const int32_t *__restrict__ nbr, int64_t nk,
                                int32_t *__restrict__ deg) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < nk) atomicAdd(&deg[nbr[e]], 1);
}

__global__ void fill_rev_kernel(const int32_t *__restrict__ nbr, int64_t nk, int k,
                                const int32_t *__restrict__ off, int32_t *__restrict__ cursor,
                                int32_t *__restrict__ src) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nk) return;
    int b = nbr[e];
    int slot = atomicAdd(&cursor[b], 1);
    src[off[b] + slot] = int32_t(e / k);
}

inline unsigned blocks_for(int64_t count, int th) { return unsigned((count + th - 1) / th); }

}  // namespace

size_t scan_workspace(int64_t count) {
    return align256(size_t((count + SCAN_TILE - 1) / SCAN_TILE + 1) * sizeof(int32_t));
}

famst_status exclusive_scan_i32(const Exec &ex, Arena &ar, const int32_t *in, int32_t *out,
                                int64_t count, int32_t *total_dev) {
    if (count <= 0) {
        if (total_dev && cudaMemsetAsync(total_dev, 0, sizeof(int32_t), ex.stream) != cudaSuccess)
            return FAMST_ERR_CUDA;
        return FAMST_OK;
    }
    int64_t nb = (count + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *bsum = ar.take<int32_t>(size_t(nb));
    if (!bsum) return FAMST_ERR_OOM;
    FAMST_LAUNCH(ex, scan_reduce_kernel, unsigned(nb), SCAN_NT, 0, in, count, bsum);
    FAMST_LAUNCH(ex, scan_blocksums_kernel, 1, 1024, 0, bsum, nb, total_dev);
    FAMST_LAUNCH(ex, scan_apply_kernel, unsigned(nb), SCAN_NT, 0, in, out, count, bsum);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

size_t radix_sort_workspace(int64_t count) {
    int64_t nb = (count + RS_TILE - 1) / RS_TILE;
    return align256(size_t(count) * 4) * 2 + align256(size_t(nb) * 256 * 4) * 2 +
           scan_workspace(nb * 256);
}

famst_status radix_sort_pairs(const Exec &ex, Arena &ar, uint32_t *keys, int32_t *vals,
                              int64_t count, int key_bits) {
    if (count <= 1 || key_bits <= 0) return FAMST_OK;
    int nb = int((count + RS_TILE - 1) / RS_TILE);
    uint32_t *k2 = ar.take<uint32_t>(size_t(count));
    int32_t *v2 = ar.take<int32_t>(size_t(count));
    int32_t *hist = ar.take<int32_t>(size_t(nb) * 256);
    int32_t *offs = ar.take<int32_t>(size_t(nb) * 256);
    if (!k2 || !v2 || !hist || !offs) return FAMST_ERR_OOM;
    uint32_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        FAMST_LAUNCH(ex, rs_hist_kernel, nb, RS_NT, 0, ka, count, shift, hist, nb);
        size_t mark = ar.off;  // the scan's scratch is reused by every pass
        famst_status st = exclusive_scan_i32(ex, ar, hist, offs, int64_t(nb) * 256, nullptr);
        ar.off = mark;
        if (st != FAMST_OK) return st;
        FAMST_LAUNCH(ex, rs_scatter_kernel, nb, RS_NT, 0, ka, va, kb, vb, count, shift, offs, nb);
        uint32_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        if (cudaMemcpyAsync(keys, ka, size_t(count) * 4, cudaMemcpyDeviceToDevice, ex.stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(vals, va, size_t(count) * 4, cudaMemcpyDeviceToDevice, ex.stream) !=
                cudaSuccess)
            return FAMST_ERR_CUDA;
    }
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

size_t components_workspace(int64_t n) {
    return align256(size_t(n) * 4) * 4 + scan_workspace(n);
}

famst_status components_uf(const Exec &ex, Arena &ar, const int32_t *nbr, int64_t n, int k,
                           int32_t *comp, int32_t *t_dev) {
    int32_t *parent = ar.take<int32_t>(size_t(n));
    int32_t *flag = ar.take<int32_t>(size_t(n));
    int32_t *rank = ar.take<int32_t>(size_t(n));
    int32_t *root = ar.take<int32_t>(size_t(n));
    if (!parent || !flag || !rank || !root) return FAMST_ERR_OOM;
    const int th = 256;
    const int lim = ex.loop_limit > 0 ? ex.loop_limit : UF_LIMIT;
    int64_t nk = n * k;
    FAMST_LAUNCH(ex, uf_init_kernel, blocks_for(n, th), th, 0, parent, n);
    if (nk > 0) {
        uint32_t vmask = 1;
        while (int64_t(vmask) + 1 < n) vmask = (vmask << 1) | 1u;
        FAMST_LAUNCH(ex, uf_hook_kernel, blocks_for((int64_t(vmask) + 1) * k, th), th, 0, nbr, n,
                     k, vmask, parent, lim, ex.dstatus);
    }
    FAMST_LAUNCH(ex, uf_flatten_kernel, blocks_for(n, th), th, 0, parent, n, root, flag, lim,
                 ex.dstatus);
    famst_status st = exclusive_scan_i32(ex, ar, flag, rank, n, t_dev);
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, uf_label_kernel, blocks_for(n, th), th, 0, root, rank, n, comp);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

size_t member_lists_workspace(int64_t n, int64_t t) {
    (void)t;
    return align256(size_t(n) * 4) + radix_sort_workspace(n);
}

famst_status member_lists(const Exec &ex, Arena &ar, const int32_t *comp, int64_t n, int64_t t,
                          int32_t *members, int32_t *comp_off) {
    uint32_t *keys = ar.take<uint32_t>(size_t(n));
    if (!keys) return FAMST_ERR_OOM;
    const int th = 256;
    FAMST_LAUNCH(ex, iota_keys_kernel, blocks_for(n, th), th, 0, comp, n, keys, members);
    int bits = 0;
    while ((int64_t(1) << bits) < t) ++bits;
    famst_status st = radix_sort_pairs(ex, ar, keys, members, n, bits);
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, segment_starts_kernel, blocks_for(n, th), th, 0, keys, n, t, comp_off);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

size_t reverse_csr_workspace(int64_t n, int k) {
    (void)k;
    return align256(size_t(n + 1) * 4) * 2 + scan_workspace(n + 1);
}

famst_status reverse_csr(const Exec &ex, Arena &ar, const int32_t *nbr, int64_t n, int k,
                         int32_t *rev_off, int32_t *rev_src) {
    int32_t *deg = ar.take<int32_t>(size_t(n + 1));
    int32_t *cursor = ar.take<int32_t>(size_t(n + 1));
    if (!deg || !cursor) return FAMST_ERR_OOM;
    const int th = 256;
    int64_t nk = n * k;
    if (cudaMemsetAsync(deg, 0, size_t(n + 1) * 4, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(cursor, 0, size_t(n + 1) * 4, ex.stream) != cudaSuccess)
        return FAMST_ERR_CUDA;
    FAMST_LAUNCH(ex, count_in_kernel, blocks_for(nk, th), th, 0, nbr, nk, deg);
    famst_status st = exclusive_scan_i32(ex, ar, deg, rev_off, n + 1, nullptr);
    if (st != FAMST_OK) return st;
    FAMST_LAUNCH(ex, fill_rev_kernel, blocks_for(nk, th), th, 0, nbr, nk, k, rev_off, cursor,
                 rev_src);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}

}  // namespace famst
