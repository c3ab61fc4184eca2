"""Parity at the full workload sizes, in the configuration bench.py times
(BF16 hi/lo distance tiles). The oracle checks what it can afford one by
one: sampled kNN rows (bit-exact), Algorithm 3 on the GPU's components
(bit-exact), Algorithm 4 on sampled edges iterated to their fixed points
(bit-exact, edges are independent), Kruskal on the GPU's full candidate
graph (identical edge set), and the gradient against the FP64 oracle."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - deselected on CPU runs
    pytest.skip("needs a CUDA device", allow_module_level=True)


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


def _check_pipeline(orc, ctx, X, k, lam, seed, n_rows, n_edges, full_refine):
    n = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    nbr_d, dist_d = ctx.knn_graph(Xd, k, "bf16x3")
    nbr, dist = nbr_d.cpu().numpy(), dist_d.cpu().numpy()
    rng = np.random.default_rng(seed)
    rows = np.concatenate([[0, n - 1], rng.choice(n, n_rows, replace=False)])
    rn, rd = orc.knn_rows(X, k, rows)
    assert np.array_equal(nbr[rows], rn) and np.array_equal(dist[rows], rd)
    # Algorithm 2 on the GPU's graph
    comp_d, t = ctx.components(nbr_d)
    G = orc.build_graph(nbr)
    C = orc.components(G)
    assert t == C.t and np.array_equal(comp_d.cpu().numpy(), C.comp)
    # Algorithm 3
    E = ctx.connect(Xd, comp_d, t, lam, seed)
    E0 = orc.random_edges(X, C, lam, seed)
    for a, b in ((E.u, E0.u), (E.v, E0.v), (E.w, E0.w), (E.ci, E0.ci), (E.cj, E0.cj)):
        assert np.array_equal(a.cpu().numpy(), b)
    # Algorithm 4
    sweeps, dh = ctx.refine(Xd, nbr_d, comp_d, E)
    if full_refine:
        Er = E0.copy()
        deltas, _ = orc.refine(X, G, C, Er)
        assert dh == deltas
    else:
        pick = rng.choice(len(E0), min(n_edges, len(E0)), replace=False)
        Er = orc.Edges(*(np.ascontiguousarray(a[pick]) for a in (E0.u, E0.v, E0.w, E0.ci, E0.cj)))
        orc.refine(X, G, C, Er)
        for a, b in ((E.u, Er.u), (E.v, Er.v), (E.w, Er.w)):
            assert np.array_equal(a.cpu().numpy()[pick], b)
        Er = orc.Edges(E.u.cpu().numpy(), E.v.cpu().numpy(), E.w.cpu().numpy(),
                       E.ci.cpu().numpy(), E.cj.cpu().numpy())
    # Kruskal-equivalent MST on the full candidate graph
    tu, tv, tw, W = ctx.mst(n, nbr_d, dist_d, E)
    T = orc.kruskal(n, nbr, dist, Er)
    assert np.array_equal(_keys(tw.cpu(), tu.cpu(), tv.cpu()), _keys(T.w, T.u, T.v))
    assert W == pytest.approx(T.W, rel=1e-12)
    return Xd, tu, tv


def test_blobs_100k_full_pipeline(orc, ctx):
    w = workloads.get("blobs_100k")
    _check_pipeline(orc, ctx, w.points(), w.k, w.lam, 11, 96, 0, full_refine=True)


@pytest.mark.slow
def test_sphere_1m_sampled_pipeline(orc, ctx):
    w = workloads.get("sphere_1m")
    _check_pipeline(orc, ctx, w.points(), w.k, w.lam, 12, 48, 4000, full_refine=False)


def test_moons_50k_backward_full(orc, ctx):
    w = workloads.get("moons_50k")
    X = w.points()
    Xd = torch.from_numpy(X).cuda()
    tree, info = ctx.build(Xd, w.k, w.lam, 1, "bf16x3")
    tu, tv = tree.u.cpu().numpy(), tree.v.cpu().numpy()
    g = ctx.mst_backward(Xd, tree.u, tree.v, 1.0).cpu().numpy()
    g64 = orc.mst_grad(X, tu, tv)
    deg = np.bincount(np.concatenate([tu, tv]), minlength=X.shape[0])[:, None]
    assert np.all(np.abs(g - g64) <= deg * (X.shape[1] + 4) * 2.0 ** -24 + 1e-7)
    # central differences (h = 1e-3) on 256 random coordinates, tree held fixed
    rng = np.random.default_rng(4)
    X64 = X.astype(np.float64)
    inc = {}
    for e, (a, b) in enumerate(zip(tu, tv)):
        inc.setdefault(int(a), []).append(e)
        inc.setdefault(int(b), []).append(e)
    h, checked = 1e-3, 0
    for _ in range(256):
        i = int(rng.integers(0, X.shape[0]))
        c = int(rng.integers(0, X.shape[1]))
        es = inc[i]
        lens = [np.sqrt(((X64[tu[e]] - X64[tv[e]]) ** 2).sum()) for e in es]
        if min(lens) < 20 * h:
            continue

        def W(delta):
            y_i = X64[i].copy()
            y_i[c] += delta
            s = 0.0
            for e in es:
                o = tv[e] if tu[e] == i else tu[e]
                s += np.sqrt(((y_i - X64[o]) ** 2).sum())
            return s
        fd = (W(h) - W(-h)) / (2 * h)
        assert abs(fd - g[i, c]) <= sum(h * h / 2 / wl ** 2 for wl in lens) + 1e-5
        checked += 1
    assert checked >= 200
