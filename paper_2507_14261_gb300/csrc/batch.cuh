// Batched build: plan (host), device buffers, enqueue (capturable).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <functional>
#include <vector>

#include "famst_internal.cuh"

namespace famst {

// Device pointers of one plan, all inside the context's batch workspace.
struct BatchDev {
    long long *voff = nullptr, *roff = nullptr, *xoff = nullptr;
    int *dims = nullptr;
    CloudDev *cl = nullptr;
    TcTile *tct = nullptr;
    F32Tile *f32t = nullptr;
    float *Xc = nullptr;
    float *Xs = nullptr;         // tensor clouds' rows in a spatial order (within each cloud)
    int32_t *perm = nullptr;     // sorted row -> compact id
    int32_t *nbr = nullptr;
    float *dist = nullptr;
    __nv_bfloat16 *H = nullptr;
    float *ny = nullptr, *xn2 = nullptr, *mean = nullptr, *splus = nullptr;
    unsigned *ymax = nullptr;
    int32_t *cand = nullptr, *fail_rows = nullptr, *fail_count = nullptr;
    int32_t *comp = nullptr, *members = nullptr, *comp_off = nullptr, *cbase = nullptr;
    uint32_t *keys = nullptr;
    long long *pp = nullptr;
    int32_t *t_dev = nullptr;
    int64_t *m_dev = nullptr, *m_req = nullptr;
    long long *tree_edges = nullptr;
    int *rounds = nullptr;
    int32_t *eu = nullptr, *ev = nullptr, *eci = nullptr, *ecj = nullptr;
    float *ew = nullptr;
    int32_t *rev_off = nullptr, *rev_src = nullptr, *hist = nullptr;
    int32_t *fu = nullptr, *fv = nullptr;
    float *fw = nullptr;
    uint32_t *tkeys = nullptr;
    int32_t *tvals = nullptr;
    double *W = nullptr;
    int32_t *f32c = nullptr, *f32fail = nullptr, *f32nfail = nullptr;  // FP32 clouds:
    float *f32w = nullptr;                      // kp candidates per row, uncertified rows
    float *Xin = nullptr;                       // copy of the caller's clouds
    int32_t *out_u = nullptr, *out_v = nullptr; // per-cloud trees before the copy out
    float *out_w = nullptr;
};

// Pinned host mirror of the results one run leaves behind.
struct BatchHost {
    double *W = nullptr;        // B
    int32_t *cbase = nullptr;   // B + 1
    int32_t *hist = nullptr;    // max_iters + 1
    int64_t *words = nullptr;   // [0] edges required, [1] forest edges, [2] rounds,
                                // [3] status word, [4] uncertified rows
};

struct BatchPlan {
    int B = 0, k = 0, lambda = 0, prec = 0, max_iters = 0;
    bool x3 = false;
    int64_t N = 0, NP = 0, m_cap = 0, tree_m = 0;
    int D = 0, max_rounds = 0;
    std::vector<long long> voff, roff, xoff;
    std::vector<int> dims;
    std::vector<CloudDev> cl;
    std::vector<TcTile> tct;
    std::vector<F32Tile> f32t;
    bool any_tc = false;
    int tc_stages = 0, tc_kc = 32, tc_epi = 4;
    size_t tc_smem = 0;
    // tile shapes the autotuner may pick from: epilogue warps, ring stages
    int n_shapes = 0, shape_epi[2] = {4, 4}, shape_stages[2] = {0, 0};
    size_t shape_smem[2] = {0, 0};
    CUtensorMap mA, mB;
    BatchDev dev;
    size_t scratch_off = 0;
};

// 1 when the tensor tiles are faster than the FP32 tiles for clouds of
// (d, n) on this device (measured once per class, cached).
int batch_autotune(const Exec &ex, int d, int64_t n, int k, bool x3);
famst_status batch_plan(const Exec &ex, const int64_t *offsets, const int32_t *dims, int B, int k,
                        int lambda, int prec, int max_iters, int64_t m_cap, BatchPlan *P);
size_t batch_workspace(const BatchPlan &P);
famst_status batch_bind(BatchPlan &P, char *base, size_t cap, cudaStream_t s);
// The captured sequence reads the clouds from dev.Xin and writes the
// trees to dev.out_*; the caller copies in and out around it.
famst_status batch_enqueue(const Exec &ex, BatchPlan &P, char *base, size_t cap, uint64_t seed,
                           BatchHost *host);
int batch_status_capacity();
// Times the batched tile pass once per tile shape on the plan's own data (the
// eager run must have prepared it) and keeps the fastest in P (cached per
// operand width, k, precision and work size).
famst_status batch_tune_tiles(const Exec &ex, BatchPlan &P);

}  // namespace famst
