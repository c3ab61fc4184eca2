"""Pins for the oracle's Algorithm 2 (components), Algorithm 3 (random
edges, Philox) and Algorithm 4 (refinement)."""
import json
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ Algorithm 2

def test_graph_is_symmetric_closure(orc):
    X = workloads.blobs(300, 5, 6, (0.3, 0.3), 11)
    nbr, _ = orc.knn(X, 3)
    G = orc.build_graph(nbr)
    want = [set() for _ in range(300)]
    for i in range(300):
        for j in nbr[i]:
            want[i].add(int(j))
            want[int(j)].add(i)
    for v in range(300):
        nb = G.neighbours(v).tolist()
        assert nb == sorted(want[v])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_components_match_scipy(orc, seed):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    X = workloads.blobs(500, 4, 12, (0.2, 0.6), seed)
    nbr, _ = orc.knn(X, 3)
    G = orc.build_graph(nbr)
    C = orc.components(G)
    n = 500
    rows = np.repeat(np.arange(n), 3)
    A = sp.csr_matrix((np.ones(n * 3), (rows, nbr.ravel())), shape=(n, n))
    t_ref, lab_ref = csgraph.connected_components(A, directed=True, connection="weak")
    assert C.t == t_ref
    # same partition
    pairs = set(zip(C.comp.tolist(), lab_ref.tolist()))
    assert len(pairs) == t_ref
    # discovery order: component c starts at its minimum id, and minima ascend
    mins = [int(C.members[C.comp_off[c]]) for c in range(C.t)]
    assert mins == sorted(mins)
    for c in range(C.t):
        mem = C.members[C.comp_off[c]:C.comp_off[c + 1]]
        assert np.all(np.diff(mem) > 0)
        assert np.all(C.comp[mem] == c)
    # every G edge joins equal components
    for v in range(n):
        assert np.all(C.comp[G.neighbours(v)] == C.comp[v])


def test_well_separated_clusters_give_at_least_cluster_count(orc):
    # centres ~65 apart in d=128 versus sigma <= 2: no kNN edge crosses
    X = workloads.blobs(1000, 128, 10, (0.5, 2.0), 4)
    nbr, _ = orc.knn(X, 5)
    C = orc.components(orc.build_graph(nbr))
    assert C.t >= 10


# ---------------------------------------------------- Philox, Algorithm 3

def test_philox_known_answers(orc):
    # known-answer vectors published with the Random123 library
    # (Salmon et al., SC'11) for Philox4x32 with 10 rounds
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        assert orc.philox4x32_10(ctr, key).tolist() == want


def test_random_edges_cross_and_are_lambda_shortest(orc):
    X = workloads.blobs(600, 6, 8, (0.2, 0.4), 21)
    nbr, _ = orc.knn(X, 4)
    G = orc.build_graph(nbr)
    C = orc.components(G)
    lam = 3
    E = orc.random_edges(X, C, lam, seed=1234)
    t = C.t
    assert t >= 8
    assert len(E) == lam * t * (t - 1) // 2
    # pair order: i outer, j inner, i < j; edge u in C_i, v in C_j
    pairs = [(i, j) for i in range(t) for j in range(i + 1, t) for _ in range(lam)]
    assert list(zip(E.ci.tolist(), E.cj.tolist())) == pairs
    assert np.all(C.comp[E.u] == E.ci) and np.all(C.comp[E.v] == E.cj)
    for e in range(len(E)):
        assert E.w[e] == orc.dist32(X[E.u[e]], X[E.v[e]])
    # within a pair the kept weights ascend
    w = E.w.reshape(-1, lam)
    assert np.all(np.diff(w, axis=1) >= 0)
    # seed changes the draw, same seed reproduces it
    E2 = orc.random_edges(X, C, lam, seed=1234)
    E3 = orc.random_edges(X, C, lam, seed=99)
    assert np.array_equal(E.u, E2.u) and np.array_equal(E.v, E2.v)
    assert not (np.array_equal(E.u, E3.u) and np.array_equal(E.v, E3.v))


def _draws_of_pair(orc, X, C, lam, seed, i, j):
    """The lambda^2 samples of component pair (i, j) regenerated here from
    the pinned Philox4x32-10 and the multiply-shift map of Alg. 3's reading
    (counter (s, p_lo, p_hi, 0), key (seed_lo, seed_hi), p = i t + j),
    as (w, s, u, v) tuples in draw order."""
    t = C.t
    p = i * t + j
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    mi = C.members[C.comp_off[i]:C.comp_off[i + 1]]
    mj = C.members[C.comp_off[j]:C.comp_off[j + 1]]
    out = []
    for s in range(lam * lam):
        r = orc.philox4x32_10([s, p & 0xFFFFFFFF, p >> 32, 0], key)
        u = int(mi[(int(r[0]) * mi.size) >> 32])
        v = int(mj[(int(r[1]) * mj.size) >> 32])
        out.append((orc.dist32(X[u], X[v]), s, u, v))
    return out


def _check_pairs_keep_lambda_smallest(orc, X, C, E, lam, seed, pairs):
    t = C.t
    discriminating = 0
    for i, j in pairs:
        draws = _draws_of_pair(orc, X, C, lam, seed, i, j)
        want = sorted(draws)[:lam]              # lambda smallest by (w, s)
        rank = i * t - i * (i + 1) // 2 + (j - i - 1)
        got = [(float(E.w[rank * lam + r]), int(E.u[rank * lam + r]), int(E.v[rank * lam + r]))
               for r in range(lam)]
        assert got == [(w, u, v) for (w, _, u, v) in want]
        # a reading that kept the first lambda draws (sorted) would differ here
        if sorted(draws[:lam]) != want:
            discriminating += 1
    return discriminating


def test_random_edges_keep_lambda_smallest_of_lambda_sq_draws(orc):
    # Alg. 3: of the lambda^2 draws of a pair, E keeps exactly the lambda
    # smallest, ordered by (w, sample index)
    X = workloads.blobs(900, 5, 9, (0.3, 0.6), 31)
    nbr, _ = orc.knn(X, 4)
    C = orc.components(orc.build_graph(nbr))
    lam, seed = 4, 0x1234_5678_9ABC
    E = orc.random_edges(X, C, lam, seed)
    t = C.t
    assert t >= 6
    pairs = [(i, j) for i in range(t) for j in range(i + 1, t)][:12]
    assert _check_pairs_keep_lambda_smallest(orc, X, C, E, lam, seed, pairs) >= 6


def test_random_edges_ties_at_lambda_th_draw_break_by_sample_index(orc):
    # integer lattice clusters: squared distances are integers, so draws of a
    # pair tie often; the lambda-th and (lambda+1)-th smallest draws tie in w
    # for some pair, and the kept one must be the one with the smaller s
    rng = np.random.default_rng(5)
    blocks = []
    for c in range(4):
        base = np.array([40 * c, 0, 0], np.float32)
        g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(2), indexing="ij"),
                     -1).reshape(-1, 3).astype(np.float32)
        blocks.append(base + g)
    X = np.ascontiguousarray(np.concatenate(blocks)[rng.permutation(128)])
    nbr, _ = orc.knn(X, 5)
    C = orc.components(orc.build_graph(nbr))
    assert C.t == 4
    lam, seed = 3, 77
    E = orc.random_edges(X, C, lam, seed)
    pairs = [(i, j) for i in range(4) for j in range(i + 1, 4)]
    _check_pairs_keep_lambda_smallest(orc, X, C, E, lam, seed, pairs)
    tied = 0
    for i, j in pairs:
        srt = sorted(_draws_of_pair(orc, X, C, lam, seed, i, j))
        if srt[lam - 1][0] == srt[lam][0]:
            tied += 1
    assert tied >= 1


def test_sample_index_mapping_is_uniform(orc):
    # multiply-shift of Philox output over a component of size 7: chi-square
    sizes = 7
    counts = np.zeros(sizes)
    for s in range(7000):
        r = orc.philox4x32_10([s, 3, 0, 0], [42, 0])
        counts[(int(r[0]) * sizes) >> 32] += 1
    chi2 = ((counts - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 22.46  # p = 0.001 for 6 degrees of freedom


def test_lambda_one_takes_single_sample(orc):
    X = workloads.blobs(300, 3, 5, (0.1, 0.1), 9)
    nbr, _ = orc.knn(X, 3)
    C = orc.components(orc.build_graph(nbr))
    E = orc.random_edges(X, C, 1, seed=7)
    assert len(E) == C.t * (C.t - 1) // 2


# ------------------------------------------------------------ Algorithm 4

def _golden_setup(orc):
    g = json.load(open(os.path.join(GOLDEN, "refine_1d.json")))
    X = np.array(g["x"], dtype=np.float32)[:, None]
    return g, X


def test_hand_worked_1d_example(orc):
    g, X = _golden_setup(orc)
    nbr, dist = orc.knn(X, g["k"])
    assert nbr.tolist() == g["knn_nbr"]
    assert dist.tolist() == g["knn_dist"]
    G = orc.build_graph(nbr)
    for v, nb in g["graph"].items():
        assert G.neighbours(int(v)).tolist() == nb
    C = orc.components(G)
    assert [C.members[C.comp_off[c]:C.comp_off[c + 1]].tolist() for c in range(C.t)] == g["components"]
    for run in g["runs"]:
        u, v, w = run["start"]
        E = orc.Edges(np.array([u], np.int32), np.array([v], np.int32),
                      np.array([w], np.float32), np.array([0], np.int32),
                      np.array([1], np.int32))
        for sweep, want_delta in zip(run["sweeps"], run["deltas"]):
            dl = orc.refine_sweep(X, G, C, E)
            assert [int(E.u[0]), int(E.v[0]), float(E.w[0])] == sweep
            assert dl == want_delta
        tree = orc.kruskal(6, nbr, dist, E)
        assert sorted(tree.w.tolist()) == g["tree_weights_sorted"]
        assert tree.W == g["W"]
        assert orc.prim_exact(X).W == g["W"]


@pytest.mark.parametrize("seed", [3, 4])
def test_refine_properties(orc, seed):
    X = workloads.blobs(800, 10, 10, (0.3, 0.8), seed)
    nbr, dist = orc.knn(X, 4)
    G = orc.build_graph(nbr)
    C = orc.components(G)
    E = orc.random_edges(X, C, 3, seed=seed)
    w0 = E.w.copy()
    deltas, changes = orc.refine(X, G, C, E)
    assert deltas[-1] == 0
    assert np.all(E.w <= w0)
    assert np.all(C.comp[E.u] == E.ci) and np.all(C.comp[E.v] == E.cj)
    # Delta of sweep s counts the edges that changed at least s times
    for s, dl in enumerate(deltas, start=1):
        assert dl == int((changes >= s).sum())
    # a fixed point: one more sweep changes nothing
    assert orc.refine_sweep(X, G, C, E) == 0
    # an edge that changed has strictly smaller weight
    assert np.all(E.w[changes > 0] < w0[changes > 0])


def test_refine_result_is_local_minimum(orc):
    # after convergence no neighbour of u improves the edge against v, and
    # no neighbour of v improves it against u (Alg. 4 fixed point)
    X = workloads.blobs(500, 4, 6, (0.3, 0.5), 8)
    nbr, _ = orc.knn(X, 3)
    G = orc.build_graph(nbr)
    C = orc.components(G)
    E = orc.random_edges(X, C, 2, seed=5)
    orc.refine(X, G, C, E)
    for e in range(len(E)):
        u, v, w = int(E.u[e]), int(E.v[e]), E.w[e]
        for up in G.neighbours(u):
            assert not orc.dist32(X[up], X[v]) < w
        for vp in G.neighbours(v):
            assert not orc.dist32(X[u], X[vp]) < w


# --------------------------------- Alg. 3 variant: the lambda nearest pairs

def test_nearest_pairs_hand_worked_1d(orc):
    g = json.load(open(os.path.join(GOLDEN, "nearest_pairs_1d.json")))
    X = np.array(g["x"], dtype=np.float32)[:, None]
    nbr, _ = orc.knn(X, g["k"])
    C = orc.components(orc.build_graph(nbr))
    assert [C.members[C.comp_off[c]:C.comp_off[c + 1]].tolist() for c in range(C.t)] == \
        g["components"]
    lam = g["lambda"]
    E = orc.nearest_edges(X, C, lam)
    assert [[int(u), int(v), float(w)] for u, v, w in zip(E.u, E.v, E.w)] == \
        [[a, b, float(w)] for a, b, w in g["kept"]]
    Eall = orc.nearest_edges(X, C, 9)   # lambda = |C_0| |C_1|: every pair, sorted
    assert [[int(u), int(v), float(w)] for u, v, w in zip(Eall.u, Eall.v, Eall.w)] == \
        [[a, b, float(w)] for a, b, w in g["all_cross_pairs_sorted"]]


def test_nearest_pairs_against_float64_cdist(orc):
    sp = pytest.importorskip("scipy.spatial")
    X = workloads.blobs(700, 7, 7, (0.3, 0.8), 17)
    nbr, _ = orc.knn(X, 4)
    C = orc.components(orc.build_graph(nbr))
    lam = 6
    E = orc.nearest_edges(X, C, lam)
    t = C.t
    assert t >= 7 and len(E) == lam * t * (t - 1) // 2
    X64 = X.astype(np.float64)
    r = 0
    for i in range(t):
        mi = C.members[C.comp_off[i]:C.comp_off[i + 1]]
        for j in range(i + 1, t):
            mj = C.members[C.comp_off[j]:C.comp_off[j + 1]]
            D = sp.distance.cdist(X64[mi], X64[mj])
            sel = slice(r * lam, (r + 1) * lam)
            u, v, w = E.u[sel], E.v[sel], E.w[sel]
            assert np.all(C.comp[u] == i) and np.all(C.comp[v] == j)
            assert np.all(E.ci[sel] == i) and np.all(E.cj[sel] == j)
            # the first kept pair is the closest pair of the two components
            assert abs(float(w[0]) - D.min()) <= 1e-5 * D.min()
            # every dropped pair is at least as far as the last kept one
            kept = set(zip(u.tolist(), v.tolist()))
            pos = {int(x): a for a, x in enumerate(mi)}
            qos = {int(x): b for b, x in enumerate(mj)}
            flat = np.sort(D, axis=None)
            assert abs(float(w[-1]) - flat[lam - 1]) <= 1e-5 * flat[lam - 1]
            for a, b in kept:
                assert abs(D[pos[a], qos[b]] - orc.dist32(X[a], X[b])) <= 1e-5 * D[pos[a], qos[b]]
            # ascending under (w, min id, max id), no pair twice
            keys = [(float(ww), min(a, b), max(a, b)) for a, b, ww in zip(u, v, w)]
            assert keys == sorted(keys) and len(set(keys)) == lam
            r += 1


def test_nearest_pairs_fewer_pairs_than_lambda_repeat_the_farthest(orc):
    g = json.load(open(os.path.join(GOLDEN, "nearest_pairs_1d.json")))
    X = np.array(g["x"], dtype=np.float32)[:, None]
    nbr, _ = orc.knn(X, g["k"])
    C = orc.components(orc.build_graph(nbr))
    E = orc.nearest_edges(X, C, 12)   # 9 cross pairs only
    got = [[int(u), int(v), float(w)] for u, v, w in zip(E.u, E.v, E.w)]
    want = [[a, b, float(w)] for a, b, w in g["all_cross_pairs_sorted"]]
    assert got == want + [want[-1]] * 3
