"""Parity of the nearest-pair variant of Algorithm 3 (famst_connect_nearest,
and famst_build with FAMST_CONNECT_NEAREST) with the oracle's brute force
over all cross pairs: the lambda nearest pairs of every component pair under
(w, min id, max id), bit-exact (ids and canonical weights), and the whole
build (tree edge set, W, sweeps) against oracle Algorithm 1 with the same
connect step."""
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


def _keys(w, u, v):
    w, u, v = (np.asarray(x) for x in (w, u, v))
    a, b = np.minimum(u, v), np.maximum(u, v)
    o = np.lexsort((b, a, w))
    return np.stack([w[o].view(np.int32).astype(np.int64), a[o], b[o]], 1)


CASES = [
    # name, cloud, k, lambda
    ("blobs_small_d16", lambda: workloads.get("blobs_small").points(), 10, 5),
    ("ragged_d3", lambda: workloads.blobs(1234, 3, 9, (0.1, 0.3), 5), 4, 7),
    ("d32_many", lambda: workloads.blobs(3001, 32, 40, (0.5, 1.5), 8), 6, 4),
    ("d77_lambda32", lambda: workloads.blobs(900, 77, 6, (0.5, 1.0), 9), 5, 32),
    ("d128", lambda: workloads.blobs(2500, 128, 12, (0.5, 2.0), 10), 8, 10),
    ("d200", lambda: workloads.blobs(1500, 200, 8, (0.5, 2.0), 11), 6, 3),
    # components of two points with k = 1: fewer cross pairs (4) than lambda
    ("tiny_components", lambda: workloads.blobs(60, 4, 30, (0.01, 0.01), 12), 1, 6),
]


@pytest.mark.parametrize("name,make,k,lam", CASES, ids=[c[0] for c in CASES])
def test_connect_nearest_matches_oracle(orc, ctx, name, make, k, lam):
    X = make()
    Xd = _dev(X)
    nbr, _ = ctx.knn_graph(Xd, k)
    comp, t = ctx.components(nbr)
    C = orc.components(orc.build_graph(nbr.cpu().numpy()))
    assert t == C.t and t >= 2
    E = ctx.connect_nearest(Xd, comp, t, lam)
    R = orc.nearest_edges(X, C, lam)
    assert len(E) == len(R) == lam * t * (t - 1) // 2
    for a, b in ((E.u, R.u), (E.v, R.v), (E.w, R.w), (E.ci, R.ci), (E.cj, R.cj)):
        assert np.array_equal(a.cpu().numpy(), b)


def test_connect_nearest_near_ties(orc, ctx):
    # every cross distance of the two shells agrees to ~1e-7 relative, far
    # inside the BF16 bounds: the canonical comparison and the (min, max)
    # tie-break decide
    rng = np.random.default_rng(4)
    a = rng.standard_normal((300, 64))
    a[:, 0] = 0.0
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = 1e-4 * rng.standard_normal((200, 64))
    b[:, 0] += 30.0
    X = np.ascontiguousarray(np.concatenate([a, b])[rng.permutation(500)], dtype=np.float32)
    Xd = _dev(X)
    nbr, _ = ctx.knn_graph(Xd, 8)
    comp, t = ctx.components(nbr)
    C = orc.components(orc.build_graph(nbr.cpu().numpy()))
    E = ctx.connect_nearest(Xd, comp, t, 12)
    R = orc.nearest_edges(X, C, 12)
    for x, y in ((E.u, R.u), (E.v, R.v), (E.w, R.w)):
        assert np.array_equal(x.cpu().numpy(), y)


@pytest.mark.parametrize("d", [16, 64, 128])
def test_build_nearest_connect_matches_oracle(orc, ctx, fam, d):
    X = workloads.blobs(2000, d, 20, (0.5, 1.5), 60 + d)
    c = fam.Context(0)
    try:
        c.set_connect_mode("nearest")
        tree, info = c.build(_dev(X), 6, 5, 3, "bf16x3")
    finally:
        c.close()
    ref = orc.famst(X, 6, 5, 3, connect="nearest")
    assert info.t == ref.C.t and info.m == len(ref.E)
    assert info.refine_sweeps == len(ref.deltas)
    assert np.array_equal(_keys(tree.w.cpu(), tree.u.cpu(), tree.v.cpu()),
                          _keys(ref.tree.w, ref.tree.u, ref.tree.v))
    assert tree.W == pytest.approx(ref.tree.W, rel=1e-12)
    # never lighter than the exact MST
    assert tree.W >= orc.prim_exact(X).W * (1 - 1e-9)


def test_connect_nearest_blobs_100k(orc, ctx):
    # the 100k x 128 mixture (50 components): all 5e9 cross pairs
    w = workloads.get("blobs_100k")
    X = w.points()
    Xd = _dev(X)
    nbr, _ = ctx.knn_graph(Xd, w.k, "bf16x3")
    comp, t = ctx.components(nbr)
    C = orc.components(orc.build_graph(nbr.cpu().numpy()))
    E = ctx.connect_nearest(Xd, comp, t, w.lam)
    R = orc.nearest_edges(X, C, w.lam)
    for a, b in ((E.u, R.u), (E.v, R.v), (E.w, R.w), (E.ci, R.ci), (E.cj, R.cj)):
        assert np.array_equal(a.cpu().numpy(), b)
