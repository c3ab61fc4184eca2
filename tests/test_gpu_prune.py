"""Phase 1 tile pruning: the kNN graph with pruning equals the graph without
it and the oracle's brute force, bit for bit, on clustered data (where most
tile pairs are skipped), on data without structure (where almost none are),
with duplicates, ragged sizes and at every precision."""
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
    c = P.Context(0)
    yield c
    c.set_knn_pruning(True)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _knn(ctx, X, k, prec, prune):
    ctx.set_knn_pruning(prune)
    nbr, dist = ctx.knn_graph(_dev(X), k, prec)
    return nbr.cpu().numpy(), dist.cpu().numpy()


CASES = [
    # name, generator, k, oracle rows (None: every row)
    ("blobs_40k_d32", lambda: workloads.blobs(40000, 32, 60, (0.5, 1.5), 31), 16, None),
    ("sphere_60k_d128", lambda: workloads.unit_sphere_mixture(60000, 128, 60, 0.02, 32), 32, 400),
    ("moons_30000_d64", lambda: workloads.get("moons_50k").points(30000), 16, 600),
    ("uniform_20k_d64", lambda: np.random.default_rng(33).random((20000, 64), np.float32), 8, None),
    ("ragged_33333_d20", lambda: workloads.blobs(33333, 20, 17, (0.3, 2.0), 34), 11, None),
    ("duplicates_24k", lambda: workloads.with_duplicates(
        workloads.blobs(20000, 16, 40, (0.5, 1.0), 35), 4000, 36), 9, None),
]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("name,make,k,rows", CASES, ids=[c[0] for c in CASES])
def test_pruned_knn_is_exact(orc, ctx, prec, name, make, k, rows):
    X = make()
    pn, pd = _knn(ctx, X, k, prec, True)
    un, ud = _knn(ctx, X, k, prec, False)
    assert np.array_equal(pn, un) and np.array_equal(pd, ud)
    if rows is None:
        rn, rd = orc.knn(X, k)
        assert np.array_equal(pn, rn) and np.array_equal(pd, rd)
    else:
        rng = np.random.default_rng(7)
        sel = np.concatenate([[0, X.shape[0] - 1], rng.choice(X.shape[0], rows, replace=False)])
        rn, rd = orc.knn_rows(X, k, sel)
        assert np.array_equal(pn[sel], rn) and np.array_equal(pd[sel], rd)


def test_pruning_skips_most_tiles_on_clusters(ctx):
    X = workloads.unit_sphere_mixture(60000, 128, 60, 0.02, 32)
    ctx.set_knn_pruning(True)
    tree, info = ctx.build(_dev(X), 32, 10, 1, "bf16x3")
    assert info.knn_tile_fraction < 0.2
    assert info.uncertified_rows == 0
    ctx.set_knn_pruning(False)
    tree0, info0 = ctx.build(_dev(X), 32, 10, 1, "bf16x3")
    assert info0.knn_tile_fraction == 1.0
    assert tree.W == tree0.W
    ctx.set_knn_pruning(True)
