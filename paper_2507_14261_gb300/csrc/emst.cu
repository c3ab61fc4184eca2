// Exact Euclidean MST of the complete graph on the GPU: the reference tree
// T* of the relative error (W_FAMST - W*) / W* of Eq. 1.
//
// Boruvka on the complete graph. Every round finds, for every point, its
// nearest neighbour outside its own current component (an exact masked
// 1-NN pass over all points, through the same distance tiles as Phase 1
// with keys of the query's own component skipped), then every component
// hooks its minimum outgoing edge under the total order (w, min id, max id).
// For one point the (w, id) order of its neighbours and the (w, min, max)
// order of its edges agree, so the component minimum is one of the
// per-point minima and each round is an exact Boruvka round. Under a strict
// total order the MST is unique: the tree equals the one Prim or Kruskal
// produce with the same weights and order.
#include "famst_internal.cuh"

namespace famst {

size_t emst_workspace(int64_t n, int d, bool tc, bool x3, int num_sms) {
    size_t knn = tc ? knn_tc_workspace(n, d, 1, x3, num_sms)
                    : knn_fp32_workspace(n, d, 1, n, num_sms);
    return boruvka_workspace(n) + align256(size_t(n) * 4) * 2 + knn;
}

famst_status emst_exact(const Exec &ex, Arena &ar, const float *X, int64_t n, int d, bool tc,
                        bool x3, bool vec4, MstOut out, int64_t *tree_edges, int *rounds,
                        int64_t *uncertified, int32_t *pin_knn, int32_t *pin_bv) {
    *tree_edges = 0;
    *rounds = 0;
    *uncertified = 0;
    if (n <= 1) return FAMST_OK;
    BvState S;
    famst_status st = bv_state_init(ex, ar, n, &S);
    if (st != FAMST_OK) return st;
    S.knn_exact = true;   // the first pass is the plain exact 1-NN
    int32_t *nbr1 = ar.take<int32_t>(size_t(n));
    float *dist1 = ar.take<float>(size_t(n));
    if (!nbr1 || !dist1) return FAMST_ERR_OOM;
    int64_t got = 0;
    // at least half the components disappear every round: 64 rounds cover any n
    for (int r = 0; r < 64 && got < n - 1; ++r) {
        const size_t mark = ar.off;
        int64_t unc = 0;
        if (tc)
            st = knn_tc(ex, ar, X, n, d, 1, x3, vec4, nbr1, dist1, pin_knn, &unc, S.comp);
        else
            st = knn_fp32(ex, ar, X, n, d, 1, nullptr, 0, n, nbr1, dist1, S.comp);
        ar.off = mark;
        if (st != FAMST_OK) return st;
        *uncertified += tc ? unc : n;
        st = bv_round(ex, ar, S, nbr1, dist1, 1, nullptr, nullptr, nullptr, 0, out, got, pin_bv);
        if (st != FAMST_OK) return st;
        *rounds = r + 1;
        const int32_t added = *pin_bv;
        if (added == 0) break;
        got += added;
    }
    *tree_edges = got;
    return FAMST_OK;
}

}  // namespace famst
