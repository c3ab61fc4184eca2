"""Parity of famst_build in the configuration bench.py times.

bench.py builds with BF16 hi/lo distance tiles (tcgen05), tile pruning on,
and Algorithm 4's kernel with its BF16 tensor-core candidate filter (the
variant a build takes for 16-byte aligned rows with 32 <= d <= 256). These
tests run exactly that call and compare the whole result with the oracle's
Algorithm 1: tree edge set (bit-exact keys), W, t, |E|, the number of
refinement sweeps and |Delta| of the first sweep. Where the oracle cannot
afford the brute-force kNN, it runs on the GPU's kNN graph after that graph
has been checked row by row against the oracle's brute force on samples
(Phase 1 is exact, so the graph is the oracle's own; a build computes it the
same way as famst_knn_graph).
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - deselected on CPU runs
    pytest.skip("needs a CUDA device", allow_module_level=True)

BF16_MMA_FILTER = 2


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_14261_gb300 as P
    return P.Context(0)


def _keys(w, u, v):
    w, u, v = (np.asarray(x) for x in (w, u, v))
    a, b = np.minimum(u, v), np.maximum(u, v)
    o = np.lexsort((b, a, w))
    return np.stack([w[o].view(np.int32).astype(np.int64), a[o], b[o]], 1)


def _compare_build(orc, ctx, X, k, lam, seed, knn_rows=None):
    """famst_build (BF16x3, pruning on) against oracle Algorithm 1. With
    knn_rows=None the oracle computes its own brute-force kNN; else it runs
    on the GPU's kNN graph, checked first on knn_rows sampled rows."""
    n = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    tree, info = ctx.build(Xd, k, lam, seed, "bf16x3")
    torch.cuda.synchronize()
    if knn_rows is None:
        ref = orc.famst(X, k, lam, seed)
    else:
        nbr_d, dist_d = ctx.knn_graph(Xd, k, "bf16x3")
        nbr, dist = nbr_d.cpu().numpy(), dist_d.cpu().numpy()
        rng = np.random.default_rng(seed)
        rows = np.concatenate([[0, n - 1], rng.choice(n, knn_rows, replace=False)])
        rn, rd = orc.knn_rows(X, k, rows)
        assert np.array_equal(nbr[rows], rn) and np.array_equal(dist[rows], rd)
        ref = orc.famst(X, k, lam, seed, knn_graph=(nbr, dist))
    assert info.t == ref.C.t
    assert info.m == len(ref.E)
    assert info.refine_sweeps == len(ref.deltas)
    if ref.deltas:
        assert info.first_delta == ref.deltas[0]
    assert np.array_equal(_keys(tree.w.cpu(), tree.u.cpu(), tree.v.cpu()),
                          _keys(ref.tree.w, ref.tree.u, ref.tree.v))
    assert tree.W == pytest.approx(ref.tree.W, rel=1e-12)
    return tree, info, ref


@pytest.mark.parametrize("d", [32, 64, 100, 128, 256])
def test_build_tensor_filter_matches_oracle(orc, ctx, d):
    # many well-separated clusters (many components, long refinement
    # trajectories), ragged n; the oracle does the full brute-force kNN
    X = workloads.blobs(3001, d, 30, (0.5, 1.5), 40 + d)
    tree, info, ref = _compare_build(orc, ctx, X, 6, 4, 9)
    assert info.t >= 30
    assert info.refine_filter == BF16_MMA_FILTER
    assert 0 < info.refine_canonical_evals < info.refine_distance_evals


def _near_tie_cloud(d, offset, seed):
    """Component A: points on a sphere of radius 1 in the hyperplane x_0 = 0
    (every one equidistant from the axis x_0), moved off it by ~1e-6; the
    other components are tight blobs (sd 1e-4) far out on the axis x_0.
    Candidate distances between the two sides then agree to about 1e-7
    relative, far inside the BF16 filter's error bound, so nearly every
    candidate goes to the canonical comparison, and FP32 ties go to the
    (w, id) tie-break. A common offset of `offset` in every coordinate adds
    the centring rounding the bounds must cover."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((400, d))
    a[:, 0] = 0.0
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    a[:, 0] = 1e-6 * rng.standard_normal(400)
    parts = [a]
    for c in range(3):
        b = 1e-4 * rng.standard_normal((200, d))
        b[:, 0] += 40.0 * (c + 1)
        parts.append(b)
    X = np.concatenate(parts) + offset
    return np.ascontiguousarray(X[rng.permutation(X.shape[0])], dtype=np.float32)


@pytest.mark.parametrize("d,offset", [(32, 0.0), (64, 1000.0), (128, 250.0)])
def test_build_filter_near_ties(orc, ctx, d, offset):
    X = _near_tie_cloud(d, offset, 3 + d)
    tree, info, ref = _compare_build(orc, ctx, X, 8, 5, 21)
    assert info.t >= 4
    assert info.refine_filter == BF16_MMA_FILTER
    # the filter could rule out few candidates here
    assert info.refine_canonical_evals > 0


def test_build_blobs_100k_matches_oracle(orc, ctx):
    w = workloads.get("blobs_100k")
    _, info, _ = _compare_build(orc, ctx, w.points(), w.k, w.lam, 1, knn_rows=64)
    assert info.refine_filter == BF16_MMA_FILTER


def test_build_sphere_200k_matches_oracle(orc, ctx):
    # the 1M x 128 sphere recipe at n = 200k: t = 1000 components and
    # lambda t (t - 1) / 2 = 4,995,000 refined edges, as in the 1M build
    w = workloads.get("sphere_1m")
    _, info, _ = _compare_build(orc, ctx, w.points(200_000), w.k, w.lam, 1, knn_rows=32)
    assert info.t == 1000 and info.refine_filter == BF16_MMA_FILTER


@pytest.mark.slow
def test_build_sphere_1m_matches_oracle(orc, ctx):
    # the benchmarked workload itself (1M x 128, k = 32, lambda = 10, seed 1)
    w = workloads.get("sphere_1m")
    _, info, _ = _compare_build(orc, ctx, w.points(), w.k, w.lam, 1, knn_rows=24)
    assert info.refine_filter == BF16_MMA_FILTER
