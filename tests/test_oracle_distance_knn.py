"""Pins for the oracle's canonical distance and its brute-force kNN."""
import numpy as np
import pytest

import workloads


def test_integer_coordinates_are_exact(orc):
    # integer coordinates with |x| <= 100 and d <= 128: every partial and
    # every butterfly sum is an integer below 2^24, so the FP32 sums are exact
    # and w must be the correctly rounded square root of the exact integer.
    rng = np.random.default_rng(5)
    for d in (1, 3, 16, 17, 128):
        a = rng.integers(-100, 101, d).astype(np.float32)
        b = rng.integers(-100, 101, d).astype(np.float32)
        exact = int(((a.astype(np.int64) - b.astype(np.int64)) ** 2).sum())
        want = np.float32(np.sqrt(np.float64(exact)))  # double sqrt rounded once more is correctly rounded
        assert orc.dist32(a, b) == want


def test_partial_sums_follow_lane_order(orc):
    # d = 64, x = 1 on coordinates 0..31 and 2^-11 on 32..63, y = 0. With the
    # partials t mod 32 every partial is 1 + 2^-22 and every butterfly sum is
    # exact, so p = 32 + 2^-17 exactly; a single running sum over t would
    # stay at 32 (each 2^-22 is below half an ulp of 32). w must be the
    # correctly rounded sqrt of the exact sum, which differs from sqrtf(32).
    a = np.concatenate([np.ones(32), np.full(32, 2.0 ** -11)]).astype(np.float32)
    b = np.zeros(64, np.float32)
    exact = np.float32(np.sqrt(np.float64(32.0) + 2.0 ** -17))
    assert exact != np.float32(np.sqrt(32.0))
    assert orc.dist32(a, b) == exact
    # the same coordinates spread so that one partial holds all the small
    # terms: 32 consecutive additions of 2^-22 to 1 + ... stay exact too
    a2 = np.zeros(64 * 32, np.float32)
    a2[0] = 1.0
    a2[32::32] = 2.0 ** -11          # partial 0 only: 1 + 63 * 2^-22, exact
    exact2 = np.float32(np.sqrt(np.float64(1.0) + 63 * 2.0 ** -22))
    assert orc.dist32(a2, np.zeros_like(a2)) == exact2


def test_distance_symmetric_bitwise(orc):
    rng = np.random.default_rng(6)
    for d in (2, 31, 64, 129):
        a = rng.standard_normal(d).astype(np.float32)
        b = rng.standard_normal(d).astype(np.float32)
        assert orc.dist32(a, b) == orc.dist32(b, a)
        assert orc.dist32(a, a) == 0.0


def test_distance_within_fp32_error_bound(orc):
    # |w32 - w| <= (gamma_{d+1}/2 + u) w  with u = 2^-24 (rounding of the
    # differences, the partial chains and the butterfly, the square root)
    rng = np.random.default_rng(7)
    u = 2.0 ** -24
    for d in (1, 5, 64, 128, 784):
        for _ in range(20):
            a = (rng.standard_normal(d) * 10).astype(np.float32)
            b = (rng.standard_normal(d) * 10).astype(np.float32)
            w64 = np.sqrt(((a.astype(np.float64) - b) ** 2).sum())
            w32 = orc.dist32(a, b)
            g = (d + 2) * u / (1 - (d + 2) * u)
            assert abs(w32 - w64) <= (g + u) * w64 + 1e-30
            assert abs(orc.dist64(a, b) - w64) <= 1e-12 * w64


def _torch_knn(X, k):
    torch = pytest.importorskip("torch")
    x = torch.from_numpy(X.astype(np.float64))
    D = torch.cdist(x, x)
    D.fill_diagonal_(float("inf"))
    vals, idx = torch.topk(D, k, dim=1, largest=False, sorted=True)
    return idx.numpy(), vals.numpy()


@pytest.mark.parametrize("n,d,k", [(300, 16, 10), (257, 3, 5), (200, 128, 16), (150, 1, 7)])
def test_knn_matches_library_float64(orc, n, d, k):
    X = workloads.blobs(n, d, centres=4, sigma=(0.5, 2.0), seed=n + d)
    nbr, dist = orc.knn(X, k)
    idx64, val64 = _torch_knn(X, k)
    # distances agree with float64 to FP32 accuracy
    assert np.allclose(dist, val64, rtol=1e-5, atol=0)
    # rows sorted by (w, id)
    for i in range(n):
        keys = list(zip(dist[i].tolist(), nbr[i].tolist()))
        assert keys == sorted(keys)
        assert i not in nbr[i]
        assert len(set(nbr[i].tolist())) == k
    # neighbour sets equal except where the k-th distance is a near tie
    mism = 0
    for i in range(n):
        if set(nbr[i]) != set(idx64[i]):
            mism += 1
            kth = val64[i, k - 1]
            # every disagreeing id lies within the FP32 tie tolerance of the k-th
            full = np.sqrt(((X.astype(np.float64) - X[i]) ** 2).sum(1))
            for j in set(nbr[i]) ^ set(idx64[i]):
                assert abs(full[j] - kth) <= 1e-5 * kth
    assert mism <= n // 20


def test_knn_brute_force_python_tiny(orc):
    rng = np.random.default_rng(8)
    X = rng.integers(-3, 4, size=(12, 2)).astype(np.float32)  # many exact ties
    k = 5
    nbr, dist = orc.knn(X, k)
    for i in range(12):
        cand = []
        for j in range(12):
            if j == i:
                continue
            w = np.float32(np.sqrt(np.float64(((X[i].astype(np.int64) - X[j].astype(np.int64)) ** 2).sum())))
            cand.append((w, j))
        cand.sort()
        assert [j for _, j in cand[:k]] == nbr[i].tolist()
        assert [w for w, _ in cand[:k]] == dist[i].tolist()


def test_knn_duplicates_are_neighbours(orc):
    X = workloads.with_duplicates(workloads.blobs(100, 8, 3, (1, 1), 1), 10, 2)
    nbr, dist = orc.knn(X, 4)
    zero_rows = np.where(dist[:, 0] == 0.0)[0]
    assert zero_rows.size >= 10
    for i in zero_rows:
        assert np.array_equal(X[nbr[i, 0]], X[i]) and nbr[i, 0] != i


def test_knn_row_ranges_and_row_lists_agree(orc):
    X = workloads.blobs(400, 12, 5, (1, 1), 3)
    a, da = orc.knn(X, 6)
    b, db = orc.knn(X, 6, rows=(100, 180))
    assert np.array_equal(a[100:180], b) and np.array_equal(da[100:180], db)
    rows = np.array([399, 0, 17, 250])
    c, dc = orc.knn_rows(X, 6, rows)
    assert np.array_equal(a[rows], c) and np.array_equal(da[rows], dc)
