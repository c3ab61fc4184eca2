"""Sizing of the pruned tile pass's split work items (host arithmetic, CPU).

A pruned Phase 1 query tile whose key list is longer than
L = max(PRUNE_SPLIT_MIN, ceil(visited / PRUNE_SPLIT_TILES)) runs as
ceil(len / L) parts; the side buffers hold PRUNE_SPLIT_SLOTS parts and the
merge grid PRUNE_SPLIT_TILES split tiles. The kernel relies on two bounds
that hold for every list-length distribution: fewer than PRUNE_SPLIT_TILES
lists are split (each has len > L and all lengths sum to visited), and their
parts number fewer than visited / L + that count, i.e. fewer than
PRUNE_SPLIT_SLOTS. This checks the bounds on adversarial distributions and
that the parts tile each list exactly, with lengths differing by at most one.
The constants are read from the header the kernels are built with.
"""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2507_14261_gb300", "csrc", "famst_internal.cuh")


def _constants():
    text = open(HDR).read()
    tiles = int(re.search(r"PRUNE_SPLIT_TILES\s*=\s*(\d+)", text).group(1))
    slots_expr = re.search(r"PRUNE_SPLIT_SLOTS\s*=\s*([^;]+);", text).group(1)
    slots = int(eval(slots_expr.replace("PRUNE_SPLIT_TILES", str(tiles))))
    mn = int(re.search(r"PRUNE_SPLIT_MIN\s*=\s*(\d+)", text).group(1))
    return tiles, slots, mn


def _split(lengths, tiles, mn):
    visited = int(lengths.sum())
    L = max(mn, -(-visited // tiles))
    parts = []
    for kt0, ln in zip(np.concatenate([[0], np.cumsum(lengths)[:-1]]), lengths):
        ln = int(ln)
        if ln > L:
            P = -(-ln // L)
            parts.append([(int(kt0) + ln * p // P, int(kt0) + ln * (p + 1) // P) for p in range(P)])
    return L, parts


def _cases(rng):
    yield "all just above the minimum", np.full(5000, 17)
    yield "one giant list", np.array([0] * 3000 + [100000] + [1] * 3000)
    yield "many lists at L + 1", np.full(20000, 33)
    yield "every list equal and long", np.full(7813, 3906)
    yield "heavy tail", rng.pareto(1.1, 8000).astype(np.int64) * 5
    yield "empty lists", np.zeros(100, np.int64)
    for t in range(20):
        nq = int(rng.integers(1, 70000))
        yield f"random {t}", rng.integers(0, int(rng.integers(1, 5000)), nq)


def test_split_counts_fit_the_buffers():
    tiles, slots, mn = _constants()
    assert slots == 2 * tiles
    rng = np.random.default_rng(2507)
    for name, lengths in _cases(rng):
        lengths = np.asarray(lengths, np.int64)
        L, parts = _split(lengths, tiles, mn)
        nsplit = len(parts)
        nparts = sum(len(p) for p in parts)
        assert nsplit < tiles or nsplit == 0, name
        assert nparts < slots or nparts == 0, name
        # only lists longer than L split; each part is non-empty, the parts
        # cover their list in order and differ in length by at most one
        offs = np.concatenate([[0], np.cumsum(lengths)])
        starts = {int(offs[q]): int(offs[q + 1]) for q in range(len(lengths)) if lengths[q] > L}
        assert len(starts) == nsplit, name
        for pl in parts:
            kt0, kt1 = pl[0][0], pl[-1][1]
            assert starts[kt0] == kt1, name
            sizes = [b - a for a, b in pl]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1, name
            assert all(pl[i][1] == pl[i + 1][0] for i in range(len(pl) - 1)), name
            assert max(sizes) <= L, name


@pytest.mark.parametrize("visited", [0, 1, 639, 640, 641, 16 * 640 + 5, 10**6, 10**9])
def test_bound_at_the_edges(visited):
    """As many lists as possible just above L, the rest of the visited
    tiles in one list that stays whole."""
    tiles, slots, mn = _constants()
    L = max(mn, -(-visited // tiles))
    m = visited // (L + 1)
    lengths = np.array([L + 1] * m + [visited - m * (L + 1)], np.int64)
    assert int(lengths.sum()) == visited
    L2, parts = _split(lengths, tiles, mn)
    assert L2 == L
    assert len(parts) == m and m < tiles
    assert sum(len(p) for p in parts) == 2 * m < slots
