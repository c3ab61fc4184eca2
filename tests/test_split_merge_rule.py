"""The rule by which the rows of a split key list are recombined (CPU).

In the pruned tile pass a row's list keeps the KC smallest scores below its
start threshold thr0 and reports KC - 1 candidates with
s+ = min(its KC-th score, thr0): a lower bound on the score of every key it
did not report, which the Phase 1 certificate relies on. When a long key
list is split, each part reports its own KC - 1 candidates and s+_p, and the
merge keeps the KC - 1 smallest over the parts' candidates with
s+ = min(the KC-th smallest of those candidates, min_p s+_p).

This checks, on random scores with many ties, that the merge gives the same
candidate scores and the same s+ as the unsplit list, and that s+ bounds the
score of every unreported key; a plausible slip (max for min, the KC-th
taken from one part) breaks one of these.
"""
import numpy as np

INF = np.float32(np.inf)


def _list(scores, ids, KC, thr0):
    """The kernel's per-row list: KC smallest scores below thr0 (+inf when
    fewer), reported as KC - 1 candidates and s+."""
    keep = scores < thr0
    s, j = scores[keep], ids[keep]
    o = np.lexsort((j, s))
    s, j = s[o][:KC], j[o][:KC]
    pad = KC - len(s)
    s = np.concatenate([s, np.full(pad, INF, np.float32)])
    j = np.concatenate([j, np.full(pad, -1)])
    return s[:KC - 1], j[:KC - 1], min(s[KC - 1], thr0)


def _merge(parts, KC):
    s = np.concatenate([p[0] for p in parts])
    j = np.concatenate([p[1] for p in parts])
    o = np.lexsort((j, s))
    s, j = s[o], j[o]
    kth = s[KC - 1] if len(s) >= KC else INF
    return s[:KC - 1], j[:KC - 1], min(kth, min(p[2] for p in parts))


def test_merge_of_parts_equals_the_unsplit_list():
    rng = np.random.default_rng(14261)
    for t in range(3000):
        KC = int(rng.choice([32, 48, 64]))
        n = int(rng.integers(1, 400))
        if t % 3 == 0:
            scores = rng.integers(-5, 6, n).astype(np.float32)      # heavy ties
        else:
            scores = rng.standard_normal(n).astype(np.float32)
        ids = rng.permutation(n)
        thr0 = INF if t % 4 == 0 else np.float32(np.quantile(scores, rng.uniform(0.05, 1.0)))
        P = int(rng.integers(2, 7))
        cuts = np.sort(rng.integers(0, n + 1, P - 1))
        bounds = np.concatenate([[0], cuts, [n]])
        parts = [_list(scores[a:b], ids[a:b], KC, thr0) for a, b in zip(bounds[:-1], bounds[1:])]
        ms, mj, msp = _merge(parts, KC)
        us, uj, usp = _list(scores, ids, KC, thr0)
        assert np.array_equal(ms, us), t
        assert msp == usp, t
        # every key not reported scores at least s+
        reported = set(int(x) for x in mj if x >= 0)
        rest = np.array([scores[q] for q in range(n) if int(ids[q]) not in reported], np.float32)
        assert rest.size == 0 or rest.min() >= msp, t
        # reported ids are distinct keys with their own scores
        sc = dict(zip(ids.tolist(), scores.tolist()))
        assert all(sc[int(x)] == float(v) for x, v in zip(mj, ms) if x >= 0), t
