// Per-thread sorted lists of the KC smallest (score, id) pairs, held in
// registers, absorbing candidates eight at a time.
//
// Inserting one candidate into a sorted register list rewrites every slot
// (a compare and four selects per slot: about 5 KC instructions). Here a
// batch of eight is first sorted (Batcher's odd-even merge sort, 19
// compare-exchanges) and then merged into the list by a bitonic merging
// network: the list followed by the reversed batch is a bitonic sequence,
// and its bitonic merge leaves the KC smallest pairs in ascending order.
// Because the list part is already sorted, most compare-exchanges of the
// textbook network are known to be no-ops and are left out: in a block whose
// first S - 8 entries are ascending, the split at distance S/2 only has to
// compare the last eight entries of each half. For KC = 48 the merge takes
// 112 compare-exchanges and 8 minima, against 8 x 48 slot updates for
// eight insertions.
//
// Any two pairs with equal scores may come out in either order; the list
// holds the KC smallest scores with ids that came in with them.
//
// Host and device: the CPU tests compile this header with a host compiler
// and check the networks exhaustively on 0-1 inputs.
#pragma once

#if defined(__CUDACC__)
#define FAMST_TOPK_HD __host__ __device__ __forceinline__
#else
#define FAMST_TOPK_HD inline
#endif

namespace famst {
namespace topk {

// compare-exchange: (as, aj) keeps the smaller score, (bs, bj) the larger
FAMST_TOPK_HD void cx(float &as, int &aj, float &bs, int &bj) {
    const bool sw = bs < as;
    const float lo = sw ? bs : as, hi = sw ? as : bs;
    const int jl = sw ? bj : aj, jh = sw ? aj : bj;
    as = lo;
    aj = jl;
    bs = hi;
    bj = jh;
}

// (as, aj) becomes the smaller of the two pairs; the larger is dropped
FAMST_TOPK_HD void keep_min(float &as, int &aj, float bs, int bj) {
    const bool sw = bs < as;
    as = sw ? bs : as;
    aj = sw ? bj : aj;
}

// eight pairs into ascending score order (Batcher's odd-even merge sort)
FAMST_TOPK_HD void sort8(float (&s)[8], int (&j)[8]) {
#define FAMST_CX(a, b) cx(s[a], j[a], s[b], j[b])
    FAMST_CX(0, 1); FAMST_CX(2, 3); FAMST_CX(4, 5); FAMST_CX(6, 7);
    FAMST_CX(0, 2); FAMST_CX(1, 3); FAMST_CX(4, 6); FAMST_CX(5, 7);
    FAMST_CX(1, 2); FAMST_CX(5, 6);
    FAMST_CX(0, 4); FAMST_CX(1, 5); FAMST_CX(2, 6); FAMST_CX(3, 7);
    FAMST_CX(2, 4); FAMST_CX(3, 5);
    FAMST_CX(1, 2); FAMST_CX(3, 4); FAMST_CX(5, 6);
#undef FAMST_CX
}

// Bitonic merge of the block [O, O + S) of (s, j), S a power of two >= 8,
// given that the block is bitonic and its first S - 8 entries ascend. The
// split at distance S/2 can only move entries whose partner lies in the
// last eight of the block (elsewhere both partners sit in the ascending
// prefix), and both halves keep the same shape.
template <int O, int S, int N>
FAMST_TOPK_HD void merge_tail8(float (&s)[N], int (&j)[N]) {
    static_assert(S >= 8 && (S & (S - 1)) == 0 && O + S <= N, "block");
    if constexpr (S == 8) {
#pragma unroll
        for (int h = 4; h >= 1; h >>= 1) {
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if ((p & h) == 0) cx(s[O + p], j[O + p], s[O + p + h], j[O + p + h]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int p = O + S / 2 - 8 + q;
            cx(s[p], j[p], s[p + S / 2], j[p + S / 2]);
        }
        merge_tail8<O, S / 2, N>(s, j);
        merge_tail8<O + S / 2, S / 2, N>(s, j);
    }
}

// (ls, lj): ascending list of KC pairs (KC = 32, 48 or 64). (bs, bj): eight
// pairs in ascending score order (+inf entries allowed). Afterwards the list
// holds the KC smallest of the KC + 8 pairs, ascending.
template <int KC>
FAMST_TOPK_HD void merge8(float (&ls)[KC], int (&lj)[KC], const float (&bs)[8],
                          const int (&bj)[8]) {
    static_assert(KC == 32 || KC == 48 || KC == 64, "list length");
    if constexpr (KC == 48) {
        // The sequence list ++ (+inf x 8) ++ reversed batch (length 64) is
        // bitonic. Distance 32: only list entries 24..31 meet batch entries.
        float us[8];
        int uj[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            us[q] = bs[7 - q];
            uj[q] = bj[7 - q];
            cx(ls[24 + q], lj[24 + q], us[q], uj[q]);
        }
        // upper half (positions 32..63): of its distance-16 split only the
        // lower block (32..47) is kept; entries 40..47 meet the batch's
        // remaining (larger) entries
#pragma unroll
        for (int q = 0; q < 8; ++q) keep_min(ls[40 + q], lj[40 + q], us[q], uj[q]);
        merge_tail8<0, 32, KC>(ls, lj);
        merge_tail8<32, 16, KC>(ls, lj);
    } else {
        // the KC smallest of list and batch: the last eight list entries
        // against the batch reversed; the result is bitonic with an
        // ascending prefix of KC - 8
#pragma unroll
        for (int q = 0; q < 8; ++q) keep_min(ls[KC - 8 + q], lj[KC - 8 + q], bs[7 - q], bj[7 - q]);
        merge_tail8<0, KC, KC>(ls, lj);
    }
}

}  // namespace topk
}  // namespace famst
