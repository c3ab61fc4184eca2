// famst_components_noalloc: connected components of the kNN graph with no
// allocation at all -- no context, no workspace, no cudaMalloc.
//
// The union-find parent array, the root flags / ranks and the per-tile
// sums of the rank scan live in one file-scope static device array of
// FAMST_NOALLOC_MAX_N-sized regions. Host code cannot pass that array's
// name to a kernel (on the host it is only a stand-in symbol), so every
// call looks up its device address in the current context with
// cudaGetSymbolAddress (nothing is cached, so a context reset leaves no
// stale address behind); every kernel receives that address.
//
// The array is shared by every call on a device and keeps the previous
// call's contents; the kernels below initialise every word they read
// (parent[v] = v, the error word = 0) before using it. Two calls whose
// work overlaps on the GPU race on the array.
#include <cuda_runtime.h>


#include "famst_internal.cuh"

namespace {

constexpr int64_t NA_MAX_N = FAMST_NOALLOC_MAX_N;
constexpr int NA_NT = 256;
constexpr int NA_IPT = 8;
constexpr int NA_TILE = NA_NT * NA_IPT;
constexpr int64_t NA_MAX_TILES = (NA_MAX_N + NA_TILE - 1) / NA_TILE;
// word offsets inside the scratch array
constexpr int64_t OFF_PARENT = 0;
constexpr int64_t OFF_RANK = NA_MAX_N;
constexpr int64_t OFF_TILES = 2 * NA_MAX_N;
constexpr int64_t OFF_WORDS = OFF_TILES + NA_MAX_TILES;  // error word, total
constexpr int64_t NA_WORDS = OFF_WORDS + 64;
constexpr int NA_LIMIT = 1 << 22;

static __device__ __align__(256) int32_t g_noalloc_scratch[NA_WORDS];

__device__ __forceinline__ int na_find(int32_t *parent_, int v, int32_t *err) {
    volatile int32_t *parent = parent_;
    int p = parent[v];
    int guard = 0;
    while (p != v) {
        if (++guard > NA_LIMIT) {
            atomicOr(err, 2);
            break;
        }
        int g = parent[p];
        if (g != p) parent[v] = g;
        v = p;
        p = g;
    }
    return v;
}

__global__ void na_init_kernel(int32_t *scratch, int64_t n) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) scratch[OFF_PARENT + v] = int32_t(v);
    if (v == 0) {
        scratch[OFF_WORDS] = 0;      // error word
        scratch[OFF_WORDS + 1] = 0;  // component count
    }
}

__global__ void na_hook_kernel(const int32_t *__restrict__ nbr, int64_t n, int k,
                               int32_t *scratch) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    int32_t *parent = scratch + OFF_PARENT;
    int32_t *err = scratch + OFF_WORDS;
    int a = int(e / k), b = nbr[e];
    if (b < 0 || int64_t(b) >= n || b == a) {  // not a kNN list of this cloud
        atomicOr(err, 1);
        return;
    }
    int ra = na_find(parent, a, err), rb = na_find(parent, b, err);
    for (int it = 0; it < NA_LIMIT; ++it) {
        if (ra == rb) return;
        int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
        int old = atomicCAS(&parent[hi], hi, lo);
        if (old == hi) return;
        if (ra > rb) ra = na_find(parent, old, err); else rb = na_find(parent, old, err);
    }
    atomicOr(err, 2);
}

// comp[v] = root of v (the smallest id of its component); rank[v] = is_root
__global__ void na_flatten_kernel(int64_t n, int32_t *scratch, int32_t *__restrict__ comp) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int r = na_find(scratch + OFF_PARENT, int(v), scratch + OFF_WORDS);
    comp[v] = r;
    scratch[OFF_RANK + v] = (r == v) ? 1 : 0;
}

__device__ int na_block_excl_scan(int v, int &total) {
    __shared__ int wsum[33];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? wsum[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wsum[32] = si;
    }
    __syncthreads();
    int excl = inc - v + wsum[w];
    total = wsum[32];
    __syncthreads();
    return excl;
}

__global__ void na_tile_sum_kernel(int64_t n, int32_t *scratch) {
    int64_t base = int64_t(blockIdx.x) * NA_TILE + int64_t(threadIdx.x) * NA_IPT;
    int s = 0;
    for (int r = 0; r < NA_IPT; ++r)
        if (base + r < n) s += scratch[OFF_RANK + base + r];
    int total;
    na_block_excl_scan(s, total);
    if (threadIdx.x == 0) scratch[OFF_TILES + blockIdx.x] = total;
}

// one block: exclusive scan of the tile sums, total = component count
__global__ void na_scan_tiles_kernel(int64_t ntiles, int32_t *scratch) {
    int carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        int v = i < ntiles ? scratch[OFF_TILES + i] : 0;
        int total;
        int excl = na_block_excl_scan(v, total);
        if (i < ntiles) scratch[OFF_TILES + i] = carry + excl;
        carry += total;
    }
    if (threadIdx.x == 0) scratch[OFF_WORDS + 1] = carry;
}

// rank[v] = number of roots below v (in place)
__global__ void na_apply_kernel(int64_t n, int32_t *scratch) {
    int64_t base = int64_t(blockIdx.x) * NA_TILE + int64_t(threadIdx.x) * NA_IPT;
    int v[NA_IPT];
    int s = 0;
    for (int r = 0; r < NA_IPT; ++r) {
        v[r] = base + r < n ? scratch[OFF_RANK + base + r] : 0;
        s += v[r];
    }
    int total;
    int run = scratch[OFF_TILES + blockIdx.x] + na_block_excl_scan(s, total);
    for (int r = 0; r < NA_IPT; ++r) {
        if (base + r < n) scratch[OFF_RANK + base + r] = run;
        run += v[r];
    }
}

__global__ void na_label_kernel(int64_t n, const int32_t *__restrict__ scratch,
                                int32_t *__restrict__ comp, int32_t *__restrict__ t_out) {
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = scratch[OFF_RANK + comp[v]];
    if (v == 0) *t_out = scratch[OFF_WORDS] ? -1 : scratch[OFF_WORDS + 1];
}

// Device address of the scratch array in the current context. Looked up on
// every call (the lookup allocates nothing): a cached address would dangle
// after cudaDeviceReset, which unloads the module with the context.
famst_status na_scratch(int32_t **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FAMST_ERR_CUDA;
    *out = static_cast<int32_t *>(p);
    return FAMST_OK;
}

inline unsigned na_blocks(int64_t count, int th) { return unsigned((count + th - 1) / th); }

}  // namespace

extern "C" famst_status famst_components_noalloc(const int32_t *nbr, int64_t n, int32_t k,
                                                 int32_t *comp, int32_t *t_dev, void *stream) {
    if (!nbr || !comp || !t_dev) return FAMST_ERR_INVALID_ARG;
    if (n < 2 || k < 1 || int64_t(k) > n - 1) return FAMST_ERR_INVALID_ARG;
    if (n > NA_MAX_N) return FAMST_ERR_UNSUPPORTED;
    if (n * int64_t(k) >= (int64_t(1) << 31)) return FAMST_ERR_UNSUPPORTED;
    int32_t *scratch = nullptr;
    famst_status st = na_scratch(&scratch);
    if (st != FAMST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int th = 256;
    const int64_t ntiles = (n + NA_TILE - 1) / NA_TILE;
    na_init_kernel<<<na_blocks(n, th), th, 0, s>>>(scratch, n);
    na_hook_kernel<<<na_blocks(n * k, th), th, 0, s>>>(nbr, n, k, scratch);
    na_flatten_kernel<<<na_blocks(n, th), th, 0, s>>>(n, scratch, comp);
    na_tile_sum_kernel<<<unsigned(ntiles), NA_NT, 0, s>>>(n, scratch);
    na_scan_tiles_kernel<<<1, 512, 0, s>>>(ntiles, scratch);
    na_apply_kernel<<<unsigned(ntiles), NA_NT, 0, s>>>(n, scratch);
    na_label_kernel<<<na_blocks(n, th), th, 0, s>>>(n, scratch, comp, t_dev);
    return cudaPeekAtLastError() == cudaSuccess ? FAMST_OK : FAMST_ERR_CUDA;
}
