"""Pins of the oracle's NN-Descent (Phase 1 as the paper runs it: an
NN-Descent library, Sec. 2 and 3; Dong, Charikar and Li, WWW 2011): a
hand-worked iteration, the exact graph as a fixed point, k = n - 1, list
invariants, monotone lists, the local-join closure of a converged graph
(every pair that met in a join can no longer improve either list), and the
recall the method is known for on clustered data."""
import json
import os

import numpy as np
import pytest

import oracle as orc
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nndescent_1d.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_nndescent_hand_worked_iteration():
    g = _golden()
    X = np.array(g["x"], np.float32)[:, None]
    r = orc.nndescent(X, g["k"], g["S"], 1, 0.0, 3, init=np.array(g["init"], np.int32))
    assert r.iters == 1
    assert r.nbr.tolist() == g["after_one"]["nbr"]
    assert r.dist.tolist() == g["after_one"]["dist"]
    assert r.updates.tolist() == g["after_one"]["updates"]
    r = orc.nndescent(X, g["k"], g["S"], 10, 0.0, 3, init=np.array(g["init"], np.int32))
    assert r.iters == g["converged"]["iters"]
    assert r.updates.tolist() == g["converged"]["updates"]
    assert r.pairs.tolist() == g["converged"]["pairs"]


def _check_lists(X, r, k):
    n = X.shape[0]
    assert r.nbr.shape == (n, k)
    for v in range(n):
        ids = r.nbr[v]
        assert len(set(ids.tolist())) == k and v not in ids and ids.min() >= 0 and ids.max() < n
        keys = list(zip(r.dist[v].tolist(), ids.tolist()))
        assert keys == sorted(keys)
        for j, w in zip(ids[:3], r.dist[v][:3]):
            assert w == orc.dist32(X[v], X[j])


def test_nndescent_lists_are_valid():
    X = workloads.blobs(700, 12, 7, (0.5, 1.5), 31)
    r = orc.nndescent(X, 9, 6, 4, 0.0, 5)
    _check_lists(X, r, 9)


def test_exact_start_is_a_fixed_point():
    X = workloads.blobs(400, 8, 4, (1.0, 1.0), 32)
    nb, dist = orc.knn(X, 6)
    r = orc.nndescent(X, 6, 6, 5, 0.0, 9, init=nb)
    assert r.iters == 1 and r.updates.tolist() == [0]
    assert np.array_equal(r.nbr, nb) and np.array_equal(r.dist, dist)


def test_k_n_minus_1_starts_exact():
    X = workloads.blobs(12, 3, 2, (1.0, 1.0), 33)
    nb, dist = orc.knn(X, 11)
    r = orc.nndescent(X, 11, 4, 3, 0.0, 1)
    assert r.updates.tolist() == [0]
    assert np.array_equal(r.nbr, nb) and np.array_equal(r.dist, dist)


def test_lists_only_improve():
    # the run with T + 1 iterations continues the one with T (same draws)
    X = workloads.blobs(900, 16, 9, (0.5, 1.5), 34)
    prev = None
    for T in range(0, 5):
        r = orc.nndescent(X, 8, 5, T, 0.0, 11)
        if prev is not None:
            assert (r.dist[:, -1] <= prev.dist[:, -1]).all()
            assert r.dist.astype(np.float64).sum() <= prev.dist.astype(np.float64).sum()
            assert r.updates[:T - 1].tolist() == prev.updates.tolist()
        prev = r


def test_converged_lists_are_closed_under_local_joins():
    # With S above every candidate count nothing is sampled away. When an
    # iteration adds nothing, every pair {a, b} of ids that share a list or
    # reverse list has met in some join, so b cannot beat B[a]'s k-th entry
    # unless it is already in B[a]. A join that skipped new x old pairs, or
    # proposed to one side only, leaves such pairs behind.
    X = workloads.blobs(300, 6, 5, (0.5, 1.0), 35)
    k = 3
    r = orc.nndescent(X, k, 32, 50, 0.0, 4)
    assert r.updates[-1] == 0
    n = X.shape[0]
    rev = [[] for _ in range(n)]
    for v in range(n):
        for u in r.nbr[v]:
            rev[u].append(v)
    assert max(k + len(x) for x in rev) <= 32   # so no candidate was sampled away
    kth = [(r.dist[a, -1], r.nbr[a, -1]) for a in range(n)]
    for v in range(n):
        cand = sorted(set(r.nbr[v].tolist()) | set(rev[v]))
        for i, a in enumerate(cand):
            for b in cand[i + 1:]:
                w = orc.dist32(X[a], X[b])
                for s, t in ((a, b), (b, a)):
                    if t not in r.nbr[s]:
                        assert (w, t) > kth[s], (v, s, t)


def test_recall_on_clusters():
    X = workloads.get("blobs_100k").points(4000)
    nb, _ = orc.knn(X, 16)
    r = orc.nndescent(X, 16, 16, 12, 0.001, 2)
    assert orc.recall(r.nbr, nb) >= 0.97
    assert orc.recall(nb, nb) == 1.0
    half = nb.copy()
    half[:, :8] = -1 - np.arange(8)   # ids no exact row holds
    assert orc.recall(half, nb) == 0.5


def test_bad_start_rows_are_rejected():
    X = workloads.blobs(20, 3, 2, (1.0, 1.0), 36)
    init = np.tile(np.arange(1, 4, dtype=np.int32), (20, 1))
    init[1] = [0, 2, 2]
    with pytest.raises(ValueError):
        orc.nndescent(X, 3, 3, 1, 0.0, 0, init=init)
