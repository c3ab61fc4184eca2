"""Pins for the oracle's Kruskal, exact Prim, the whole of Algorithm 1, and
the gradient of the tree weight."""
import itertools

import numpy as np
import pytest

import workloads


def _is_spanning_tree(n, u, v):
    if len(u) != n - 1:
        return False
    par = list(range(n))

    def f(x):
        while par[x] != x:
            par[x] = par[par[x]]
            x = par[x]
        return x
    for a, b in zip(u, v):
        ra, rb = f(int(a)), f(int(b))
        if ra == rb:
            return False
        par[ra] = rb
    return True


def _key_list(w, u, v):
    return sorted((float(a), min(int(b), int(c)), max(int(b), int(c))) for a, b, c in zip(w, u, v))


@pytest.mark.parametrize("seed", range(4))
def test_prim_and_kruskal_match_enumeration(orc, seed):
    rng = np.random.default_rng(seed)
    n = 7
    # small integer coordinates: many exact ties exercise the total order
    X = rng.integers(0, 3, size=(n, 2)).astype(np.float32)
    X[:, 1] += np.arange(n) % 2
    pairs = list(itertools.combinations(range(n), 2))
    w = {p: orc.dist32(X[p[0]], X[p[1]]) for p in pairs}
    best = None
    for sub in itertools.combinations(pairs, n - 1):
        if not _is_spanning_tree(n, [a for a, _ in sub], [b for _, b in sub]):
            continue
        keys = sorted((w[p], p[0], p[1]) for p in sub)
        W = sum(float(k[0]) for k in keys)
        cand = (W, keys)
        if best is None or cand < best:
            best = cand
    prim = orc.prim_exact(X)
    # Kruskal on the complete graph given as k = n-1 neighbour lists
    nbr, dist = orc.knn(X, n - 1)
    kr = orc.kruskal(n, nbr, dist, None)
    for T in (prim, kr):
        assert abs(T.W - best[0]) <= 1e-9
        assert _key_list(T.w, T.u, T.v) == [(float(a), b, c) for a, b, c in best[1]]


def test_kruskal_matches_scipy_on_sparse_graphs(orc):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for seed in range(3):
        X = workloads.blobs(400, 6, 1, (1, 1), seed)
        nbr, dist = orc.knn(X, 8)
        n = 400
        rows = np.repeat(np.arange(n), 8)
        A = sp.coo_matrix((dist.ravel().astype(np.float64), (rows, nbr.ravel())), shape=(n, n)).tocsr()
        A = A.maximum(A.T)
        ref = csgraph.minimum_spanning_tree(A)
        ncomp, _ = csgraph.connected_components(A, directed=False)
        T = orc.kruskal(n, nbr, dist, None)
        assert len(T.u) == n - ncomp
        assert abs(T.W - ref.sum()) <= 1e-9 * T.W


def test_closed_forms(orc):
    # collinear integer points: W = max - min
    X = workloads.collinear(60, 3, seed=1)
    T = orc.prim_exact(X)
    assert T.W == float(X[:, 0].max() - X[:, 0].min())
    r = orc.famst(X, k=2, lam=2, seed=3)
    assert r.tree.W >= T.W
    # unit m x m grid: W = m^2 - 1, every tree edge has length 1
    for m in (3, 6):
        G = workloads.integer_grid(m, d=4)
        T = orc.prim_exact(G)
        assert T.W == m * m - 1 and np.all(T.w == 1.0)
    # regular polygon: W = (n-1) * side
    P = workloads.regular_polygon(13, radius=5.0)
    T = orc.prim_exact(P)
    side = 2 * 5.0 * np.sin(np.pi / 13)
    assert abs(T.W - 12 * side) <= 12 * side * 1e-6


@pytest.mark.parametrize("n,d", [(40, 3), (64, 16)])
def test_k_equal_n_minus_1_is_exact(orc, n, d):
    X = workloads.blobs(n, d, 3, (1, 1), n)
    r = orc.famst(X, k=n - 1, lam=3, seed=1)
    assert r.C.t == 1 and len(r.E) == 0
    P = orc.prim_exact(X)
    assert r.tree.key_sorted()[1].tolist() == P.key_sorted()[1].tolist()
    assert r.tree.key_sorted()[2].tolist() == P.key_sorted()[2].tolist()
    assert r.tree.W == pytest.approx(P.W, rel=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_famst_tree_is_spanning_and_not_lighter_than_exact(orc, seed):
    X = workloads.blobs(600, 8, 9, (0.3, 1.0), seed)
    r = orc.famst(X, k=5, lam=3, seed=seed)
    T = r.tree
    assert _is_spanning_tree(600, T.u, T.v)
    P = orc.prim_exact(X)
    assert T.W >= P.W - 1e-9 * P.W
    err = orc.relative_error(T.W, P.W)
    assert 0 <= err < 0.05
    # the tree uses only candidate edges: kNN edges or refined E edges
    cand = set()
    for i in range(600):
        for j in r.nbr[i]:
            cand.add((min(i, int(j)), max(i, int(j))))
    for a, b in zip(r.E.u, r.E.v):
        cand.add((min(int(a), int(b)), max(int(a), int(b))))
    for a, b in zip(T.u, T.v):
        assert (int(a), int(b)) in cand


def test_single_point_and_two_points(orc):
    T = orc.prim_exact(np.zeros((1, 3), np.float32))
    assert T.W == 0.0 and len(T.u) == 0
    X = np.array([[0, 0], [3, 4]], np.float32)
    r = orc.famst(X, k=1, lam=1, seed=0)
    assert r.tree.W == 5.0


# ---------------------------------------------------------------- gradient

def test_gradient_two_points_closed_form(orc):
    X = np.array([[1.0, 2.0, 2.0], [0.0, 0.0, 0.0]], np.float32)
    g = orc.mst_grad(X, np.array([0]), np.array([1]))
    assert np.allclose(g[0], np.array([1, 2, 2]) / 3.0, rtol=0, atol=1e-15)
    assert np.allclose(g[1], -g[0], rtol=0, atol=0)


def test_gradient_matches_central_differences(orc):
    X = workloads.two_moons(200, 6, noise=0.05, seed=2)
    r = orc.famst(X, k=6, lam=2, seed=1)
    tu, tv = r.tree.u, r.tree.v
    g = orc.mst_grad(X, tu, tv)
    Xd = X.astype(np.float64)
    # central differences in double; h small enough that the O(h^2 / w^2)
    # truncation term is far below the tolerance for edges of length ~1e-2
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(40):
        i = int(rng.integers(0, 200))
        c = int(rng.integers(0, 6))
        # W with the tree held fixed, only edges at i change
        inc = [(a, b) for a, b in zip(tu, tv) if a == i or b == i]

        def W(delta):
            y = Xd.copy()
            y[i, c] += delta
            return sum(np.sqrt(((y[a] - y[b]) ** 2).sum()) for a, b in inc)
        fd = (W(h) - W(-h)) / (2 * h)
        assert abs(fd - g[i, c]) <= 1e-6 * max(1.0, abs(g[i, c]))
