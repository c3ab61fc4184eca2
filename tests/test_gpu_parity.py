"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every distance is the canonical FP32 distance on both sides, so kNN lists,
component labels, inter-component edges, refined edges and tree edge sets
must be bit-identical; tree weights (FP64 sums in different orders) agree to
1e-12 relative. The gradient is FP32 on the GPU and FP64 in the oracle.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - deselected on CPU runs
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def fam():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_14261_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(fam):
    return fam.Context(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _tree_keys(w, u, v):
    w, u, v = (np.asarray(x) for x in (w, u, v))
    a, b = np.minimum(u, v), np.maximum(u, v)
    return sorted(zip(w.tolist(), a.tolist(), b.tolist()))


KNN_CASES = [
    ("blobs_small", lambda: workloads.get("blobs_small").points(), 10),
    ("ragged_257x17", lambda: workloads.blobs(257, 17, 5, (0.5, 2.0), 3), 7),
    ("d1", lambda: workloads.blobs(300, 1, 4, (1, 1), 4), 5),
    ("k128", lambda: workloads.blobs(700, 8, 3, (1, 1), 5), 128),
    ("k_n_minus_1", lambda: workloads.blobs(40, 3, 2, (1, 1), 6), 39),
    ("grid_ties", lambda: workloads.integer_grid(20, d=5), 12),
    ("duplicates", lambda: workloads.with_duplicates(workloads.blobs(500, 32, 4, (1, 1), 7), 40, 8), 9),
    ("d129", lambda: workloads.blobs(1100, 129, 6, (0.5, 2.0), 9), 16),
]


@pytest.mark.parametrize("name,make,k", KNN_CASES, ids=[c[0] for c in KNN_CASES])
def test_knn_fp32_exact(orc, ctx, name, make, k):
    X = make()
    nbr, dist = ctx.knn_graph(_dev(X), k, "fp32")
    rn, rd = orc.knn(X, k)
    assert np.array_equal(nbr.cpu().numpy(), rn)
    assert np.array_equal(dist.cpu().numpy(), rd)


def _oracle_stages(orc, X, nbr, lam, seed):
    G = orc.build_graph(nbr)
    C = orc.components(G)
    E0 = orc.random_edges(X, C, lam, seed)
    return G, C, E0


@pytest.mark.parametrize("wl,n", [("blobs_small", None), ("moons_50k", 3000)])
def test_phase_by_phase(orc, ctx, wl, n):
    w = workloads.get(wl)
    X = w.points(n)
    k, lam, seed = w.k, w.lam, 1234
    Xd = _dev(X)
    nbr, dist = ctx.knn_graph(Xd, k)
    rn, rd = orc.knn(X, k)
    assert np.array_equal(nbr.cpu().numpy(), rn) and np.array_equal(dist.cpu().numpy(), rd)
    # Alg. 2
    comp, t = ctx.components(nbr)
    G, C, E0 = _oracle_stages(orc, X, rn, lam, seed)
    assert t == C.t
    assert np.array_equal(comp.cpu().numpy(), C.comp)
    # Alg. 3
    E = ctx.connect(Xd, comp, t, lam, seed)
    assert len(E) == len(E0)
    for a, b in ((E.u, E0.u), (E.v, E0.v), (E.w, E0.w), (E.ci, E0.ci), (E.cj, E0.cj)):
        assert np.array_equal(a.cpu().numpy(), b)
    # Alg. 4
    Er = E0.copy()
    deltas, _ = orc.refine(X, G, C, Er)
    sweeps, dh = ctx.refine(Xd, nbr, comp, E)
    assert sweeps == len(deltas) and dh == deltas
    for a, b in ((E.u, Er.u), (E.v, Er.v), (E.w, Er.w)):
        assert np.array_equal(a.cpu().numpy(), b)
    # Kruskal-equivalent MST
    tu, tv, tw, W = ctx.mst(X.shape[0], nbr, dist, E)
    T = orc.kruskal(X.shape[0], rn, rd, Er)
    assert _tree_keys(tw.cpu(), tu.cpu(), tv.cpu()) == _tree_keys(T.w, T.u, T.v)
    assert W == pytest.approx(T.W, rel=1e-12)
    W2, W64 = ctx.tree_weight(Xd, tu, tv, tw)
    assert W2 == W
    assert W64 == pytest.approx(orc.tree_weight64(X, T.u, T.v), rel=1e-12)


@pytest.mark.parametrize("seed", [0, 5])
def test_build_matches_oracle(orc, ctx, seed):
    X = workloads.get("blobs_small").points()
    tree, info = ctx.build(_dev(X), 10, 5, seed)
    ref = orc.famst(X, 10, 5, seed)
    assert _tree_keys(tree.w.cpu(), tree.u.cpu(), tree.v.cpu()) == \
        _tree_keys(ref.tree.w, ref.tree.u, ref.tree.v)
    assert tree.W == pytest.approx(ref.tree.W, rel=1e-12)
    assert info.t == ref.C.t and info.m == len(ref.E)
    assert info.refine_sweeps == len(ref.deltas)
    assert info.first_delta == ref.deltas[0]
    # exact MST for Eq. 1: the approximate tree is never lighter
    P = orc.prim_exact(X)
    assert tree.W >= P.W - 1e-9 * P.W
    assert info.W64 == pytest.approx(orc.tree_weight64(X, ref.tree.u, ref.tree.v), rel=1e-12)


def test_k_n_minus_1_gives_exact_mst(orc, ctx):
    X = workloads.blobs(90, 6, 3, (1, 1), 12)
    tree, info = ctx.build(_dev(X), 89, 3, 0)
    assert info.t == 1 and info.m == 0
    P = orc.prim_exact(X)
    assert _tree_keys(tree.w.cpu(), tree.u.cpu(), tree.v.cpu()) == _tree_keys(P.w, P.u, P.v)


def test_closed_forms_on_gpu(ctx):
    X = workloads.collinear(500, 4, seed=3)
    tree, _ = ctx.build(_dev(X), 2, 2, 1)
    assert tree.W >= float(X[:, 0].max() - X[:, 0].min())
    G = workloads.integer_grid(30, d=3)
    tree, info = ctx.build(_dev(G), 4, 2, 1)
    assert tree.W == 30 * 30 - 1 and np.all(tree.w.cpu().numpy() == 1.0)


def test_hand_worked_example_on_gpu(ctx):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "refine_1d.json")))
    X = np.array(g["x"], np.float32)[:, None]
    Xd = _dev(X)
    nbr, dist = ctx.knn_graph(Xd, 1)
    assert nbr.cpu().numpy().tolist() == g["knn_nbr"]
    comp, t = ctx.components(nbr)
    assert t == 2
    import paper_2507_14261_gb300 as P
    for run in g["runs"]:
        u, v, w = run["start"]
        E = P.Edges(*(torch.tensor([a], dtype=dt, device="cuda") for a, dt in
                      ((u, torch.int32), (v, torch.int32), (w, torch.float32), (0, torch.int32),
                       (1, torch.int32))))
        sweeps, dh = ctx.refine(Xd, nbr, comp, E)
        assert [int(E.u[0]), int(E.v[0]), float(E.w[0])] == run["sweeps"][-1]
        assert dh == run["deltas"] and sweeps == len(run["deltas"])
    tree, _ = ctx.build(Xd, 1, 1, 0)
    assert tree.W == g["W"]


def test_single_point_and_pairs(ctx):
    import paper_2507_14261_gb300 as P
    X = torch.zeros((1, 3), device="cuda")
    tree, info = ctx.build(X, 1, 1)
    assert tree.W == 0.0
    X = torch.tensor([[0.0, 0.0], [3.0, 4.0]], device="cuda")
    tree, info = ctx.build(X, 1, 1)
    assert tree.W == 5.0
    del P


# ------------------------------------------------------------- backward

def test_backward_matches_fp64_oracle_and_fd(orc, ctx):
    w = workloads.get("moons_50k")
    X = w.points(4000)
    Xd = _dev(X)
    tree, _ = ctx.build(Xd, w.k, w.lam, 1)
    tu, tv = tree.u.cpu().numpy(), tree.v.cpu().numpy()
    g = ctx.mst_backward(Xd, tree.u, tree.v, 1.0).cpu().numpy()
    g64 = orc.mst_grad(X, tu, tv)
    # FP32 terms (x_i - x_j)/w_ij of magnitude <= 1, summed over a vertex's
    # tree edges: |error| <= deg * (d + 4) * 2^-24 per component
    deg = np.bincount(np.concatenate([tu, tv]), minlength=X.shape[0])[:, None]
    assert np.all(np.abs(g - g64) <= deg * (X.shape[1] + 4) * 2.0 ** -24 + 1e-7)
    # central differences with the tree held fixed (h = 1e-3)
    rng = np.random.default_rng(0)
    Xd64 = X.astype(np.float64)
    for _ in range(32):
        i = int(rng.integers(0, X.shape[0]))
        c = int(rng.integers(0, X.shape[1]))
        inc = [(a, b) for a, b in zip(tu, tv) if a == i or b == i]

        def W(delta):
            y = Xd64.copy()
            y[i, c] += delta
            return sum(np.sqrt(((y[a] - y[b]) ** 2).sum()) for a, b in inc)
        h = 1e-3
        fd = (W(h) - W(-h)) / (2 * h)
        # truncation error of central differences is h^2/6 * |W'''| with
        # |W'''| <= 3 / min edge length^2 over the incident edges
        lens = [np.sqrt(((Xd64[a] - Xd64[b]) ** 2).sum()) for a, b in inc]
        if min(lens) < 20 * h:
            continue  # too close to the kink of |x| at 0 for this step
        bound = sum(h * h / 2 / wl ** 2 for wl in lens)
        assert abs(fd - g[i, c]) <= bound + 1e-5


def test_autograd_function(orc, fam):
    X = torch.from_numpy(workloads.blobs(800, 8, 4, (1, 1), 2)).cuda().requires_grad_(True)
    W = fam.mst_weight(X, 8, 3, 5)
    W.backward()
    ref = orc.famst(X.detach().cpu().numpy(), 8, 3, 5)
    assert float(W) == pytest.approx(ref.tree.W, rel=1e-12)
    g64 = orc.mst_grad(X.detach().cpu().numpy(), ref.tree.u, ref.tree.v)
    assert np.allclose(X.grad.cpu().numpy(), g64, rtol=1e-4, atol=1e-5)


# ------------------------------------------------------ error handling

def test_errors_are_reported(ctx, fam):
    X = workloads.blobs(200, 4, 3, (1, 1), 1)
    Xd = _dev(X)
    with pytest.raises(fam.FamstError) as e:
        ctx.knn_graph(Xd, 200)
    assert e.value.name == "FAMST_ERR_INVALID_ARG"
    Xn = Xd.clone()
    Xn[17, 2] = float("nan")
    with pytest.raises(fam.FamstError) as e:
        ctx.build(Xn, 5, 2)
    assert e.value.name == "FAMST_ERR_NONFINITE"
    Xi = Xd.clone()
    Xi[3, 0] = float("inf")
    with pytest.raises(fam.FamstError) as e:
        ctx.knn_graph(Xi, 5)
    assert e.value.name == "FAMST_ERR_NONFINITE"
    nbr, dist = ctx.knn_graph(Xd, 3)
    comp, t = ctx.components(nbr)
    assert t >= 2
    with pytest.raises(fam.FamstError) as e:
        ctx.connect(Xd, comp, t, 3, 1, capacity=1)
    assert e.value.name == "FAMST_ERR_CAPACITY"
    bad = nbr.clone()
    bad[5, 1] = 10_000
    with pytest.raises(fam.FamstError) as e:
        ctx.components(bad)
    assert e.value.name == "FAMST_ERR_INVALID_ARG"
    # the context stays usable after errors
    nbr2, _ = ctx.knn_graph(Xd, 3)
    assert torch.equal(nbr, nbr2)


def test_refine_iteration_cap(orc, ctx, fam):
    # start every edge from its worst sample so it must move at least once
    X = workloads.blobs(1500, 8, 8, (0.5, 0.5), 3)
    Xd = _dev(X)
    nbr, dist = ctx.knn_graph(Xd, 4)
    comp, t = ctx.components(nbr)
    E = ctx.connect(Xd, comp, t, 2, 9)
    E2 = E.clone()
    sweeps, dh = ctx.refine(Xd, nbr, comp, E)
    assert sweeps >= 2
    with pytest.raises(fam.FamstError) as e:
        ctx.refine(Xd, nbr, comp, E2, max_iters=sweeps - 1)
    assert e.value.name == "FAMST_ERR_NO_CONVERGENCE"


def test_loop_limit_reports_timeout_and_context_recovers(orc, ctx, fam):
    # evenly spaced collinear points with k = 2: the kNN graph is one long
    # path, so the union-find trees are deep and Boruvka needs many rounds; a
    # limit of one step / one round must end each call with
    # FAMST_ERR_TIMEOUT (a status the bounded loops raise, no fault), and the
    # context must work after
    n = 3000
    X = np.zeros((n, 4), np.float32)
    X[:, 0] = np.random.default_rng(3).permutation(n)   # unit spacing, shuffled ids
    Xd = _dev(X)
    nbr, dist = ctx.knn_graph(Xd, 2)
    comp_ref, t_ref = ctx.components(nbr)
    assert t_ref == 1
    try:
        ctx.set_loop_limit(1)
        with pytest.raises(fam.FamstError) as e:
            ctx.components(nbr)
        assert e.value.name == "FAMST_ERR_TIMEOUT"
        with pytest.raises(fam.FamstError) as e:
            ctx.mst(n, nbr, dist, None)
        assert e.value.name == "FAMST_ERR_TIMEOUT"
        with pytest.raises(fam.FamstError) as e:
            ctx.build(Xd, 2, 2, 1)
        assert e.value.name == "FAMST_ERR_TIMEOUT"
    finally:
        ctx.set_loop_limit(0)
    comp, t = ctx.components(nbr)
    assert t == 1 and torch.equal(comp, comp_ref)
    tu, tv, tw, W = ctx.mst(n, nbr, dist, None)
    T = orc.kruskal(n, nbr.cpu().numpy(), dist.cpu().numpy(), None)
    assert _tree_keys(tw.cpu(), tu.cpu(), tv.cpu()) == _tree_keys(T.w, T.u, T.v)
    assert W == n - 1


def test_workspace_query_matches_a_build(fam):
    # a fresh context grows its workspace to exactly what the query reports
    # (plus the quarter of slack each slot is allocated with)
    w = workloads.get("blobs_100k")
    X = w.points(20_000)
    c = fam.Context(0)
    try:
        tree, info = c.build(_dev(X), w.k, w.lam, 1, "bf16x3")
        q = c.workspace_query(X.shape[0], X.shape[1], w.k, w.lam, info.t, "bf16x3")
        held = c.workspace_bytes
        assert q <= held <= q + q // 4 + 16
        # more components can only need more
        assert c.workspace_query(X.shape[0], X.shape[1], w.k, w.lam, 4 * info.t, "bf16x3") > q
        with pytest.raises(fam.FamstError):
            c.workspace_query(X.shape[0], X.shape[1], w.k, w.lam, 0, "bf16x3")
    finally:
        c.close()
