"""Parity of the tcgen05 (BF16 / BF16 hi-lo x3 / E4M3) distance path with the
oracle's exact kNN: candidates from reduced-precision tiles, canonical FP32
re-rank, certificate, FP32 recomputation of uncertified rows -- the output
must equal the brute-force kNN bit for bit, at any precision."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    # name, generator, k
    ("blobs_small", lambda: workloads.get("blobs_small").points(), 10),
    ("blobs_100k_recipe_3000", lambda: workloads.get("blobs_100k").points(3000), 16),
    ("sphere_recipe_5000", lambda: workloads.unit_sphere_mixture(5000, 128, 5, 0.02, 2), 32),
    ("moons_recipe_2000", lambda: workloads.get("moons_50k").points(2000), 16),
    ("ragged_1037x77", lambda: workloads.blobs(1037, 77, 7, (0.5, 2.0), 4), 9),
    ("d3", lambda: workloads.blobs(900, 3, 6, (1.0, 1.0), 5), 16),
    ("d129", lambda: workloads.blobs(1300, 129, 6, (0.5, 2.0), 6), 31),
    ("k1", lambda: workloads.blobs(600, 32, 4, (1.0, 1.0), 7), 1),
    ("k63", lambda: workloads.blobs(2100, 24, 4, (1.0, 1.0), 8), 63),
    ("grid_ties", lambda: workloads.integer_grid(24, d=8), 12),
    ("duplicates", lambda: workloads.with_duplicates(workloads.blobs(800, 16, 4, (1, 1), 9), 60, 10), 8),
    ("tiny_n", lambda: workloads.blobs(20, 8, 2, (1, 1), 11), 19),
]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "fp8"])
@pytest.mark.parametrize("name,make,k", CASES, ids=[c[0] for c in CASES])
def test_tensor_knn_is_exact(orc, ctx, prec, name, make, k):
    X = make()
    nbr, dist = ctx.knn_graph(_dev(X), k, prec)
    rn, rd = orc.knn(X, k)
    assert np.array_equal(nbr.cpu().numpy(), rn)
    assert np.array_equal(dist.cpu().numpy(), rd)


def test_x3_certifies_well_conditioned_rows(ctx):
    # the hi/lo split keeps the score error near 2^-16 |x||y|: on the
    # clustered recipes nearly every row is certified without recomputation
    for X, k in ((workloads.get("blobs_100k").points(6000), 16),
                 (workloads.unit_sphere_mixture(8000, 128, 8, 0.02, 3), 32)):
        tree, info = ctx.build(_dev(X), k, 3, 1, "bf16x3")
        assert info.uncertified_rows <= X.shape[0] // 100


def test_build_matches_fp32_path(ctx):
    X = workloads.get("blobs_100k").points(5000)
    Xd = _dev(X)
    t32, i32 = ctx.build(Xd, 16, 5, 3, "fp32")
    for prec in ("bf16x3", "bf16", "fp8"):
        t, i = ctx.build(Xd, 16, 5, 3, prec)
        assert torch.equal(t.u, t32.u) and torch.equal(t.v, t32.v) and torch.equal(t.w, t32.w)
        assert t.W == t32.W


def _separated_groups(groups, size, d, seed):
    # groups of `size` points (spread 0.01) whose centres are >= 10 apart:
    # for k < size the k-th neighbour lies in the point's own group and every
    # point outside it is ~1000x farther, a gap far above E4M3's 2^-4 error
    rng = np.random.default_rng(seed)
    c = 10.0 * np.eye(groups, d) if groups <= d else 10.0 * rng.standard_normal((groups, d))
    X = np.repeat(c, size, axis=0) + 0.01 * rng.standard_normal((groups * size, d))
    return np.ascontiguousarray(X[rng.permutation(len(X))], dtype=np.float32)


def test_fp8_certifies_separated_groups(orc, ctx):
    X = _separated_groups(128, 24, 128, 21)
    tree, info = ctx.build(_dev(X), 10, 3, 1, "fp8")
    assert info.uncertified_rows <= X.shape[0] // 100
    nbr, dist = ctx.knn_graph(_dev(X), 10, "fp8")
    rn, rd = orc.knn(X, 10)
    assert np.array_equal(nbr.cpu().numpy(), rn) and np.array_equal(dist.cpu().numpy(), rd)


def test_fp8_scales_span_magnitudes(orc, ctx):
    # rows from 1e-6 to 1e6 in norm: each row's power-of-two scale keeps its
    # E4M3 codes in range, and the exact result does not depend on it
    rng = np.random.default_rng(5)
    X = rng.standard_normal((1500, 40)) * np.exp(rng.uniform(-14, 14, (1500, 1)))
    X = np.ascontiguousarray(X, dtype=np.float32)
    nbr, dist = ctx.knn_graph(_dev(X), 7, "fp8")
    rn, rd = orc.knn(X, 7)
    assert np.array_equal(nbr.cpu().numpy(), rn) and np.array_equal(dist.cpu().numpy(), rd)


def test_fp8_only_where_supported(ctx):
    import paper_2507_14261_gb300 as P
    X = _dev(workloads.blobs(500, 16, 4, (1, 1), 3))
    with pytest.raises(P.FamstError) as e:
        ctx.emst_exact(X, "fp8")
    assert e.value.name == "FAMST_ERR_UNSUPPORTED"
    with pytest.raises(P.FamstError) as e:
        ctx.build_batched(X.reshape(-1), [0, 500], [16], 5, 3, 1, "fp8")
    assert e.value.name == "FAMST_ERR_UNSUPPORTED"
