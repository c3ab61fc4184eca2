"""The register top-KC list networks of the tile kernel's epilogue
(csrc/topk_merge.cuh), compiled for the host and checked on the CPU.

The tile kernel keeps, for every query row, the KC smallest scores seen so
far (Phase 1 of Algorithm 1: the k nearest neighbours plus slack for the
certificate). It absorbs candidates eight at a time: a sorting network for
the batch, then a bitonic merge with the list that leaves out compare-
exchanges known to be no-ops on a sorted list. Both are comparator networks
on inputs from a class closed under monotone maps (a sorted list and a
batch), so by the 0-1 principle an exhaustive check on 0-1 inputs proves
them for all inputs; random float cases with ties and +inf also check that
every output pair is an input pair (ids travel with their scores).
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2507_14261_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <algorithm>
#include <vector>
#include <random>
#include <utility>
#include "topk_merge.cuh"
using namespace famst::topk;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails < 10) { std::printf(__VA_ARGS__); std::printf("\n"); } ++fails; } } while (0)

static void test_sort8() {
    for (int m = 0; m < 256; ++m) {              // every 0-1 input
        float s[8]; int j[8];
        for (int c = 0; c < 8; ++c) { s[c] = float((m >> c) & 1); j[c] = c; }
        sort8(s, j);
        int ones = __builtin_popcount(m);
        for (int c = 0; c < 8; ++c) CHECK(s[c] == (c >= 8 - ones ? 1.f : 0.f), "sort8 0-1 m=%d", m);
        bool seen[8] = {};
        for (int c = 0; c < 8; ++c) { CHECK(s[c] == float((m >> j[c]) & 1), "sort8 id"); seen[j[c]] = true; }
        for (int c = 0; c < 8; ++c) CHECK(seen[c], "sort8 perm");
    }
}

template <int KC>
static void test_merge01() {
    // list: KC - a zeros then ones; batch: b zeros then ones (both ascending)
    for (int a = 0; a <= KC; ++a)
        for (int b = 0; b <= 8; ++b) {
            float ls[KC]; int lj[KC]; float bs[8]; int bj[8];
            for (int p = 0; p < KC; ++p) { ls[p] = p < a ? 0.f : 1.f; lj[p] = p; }
            for (int c = 0; c < 8; ++c) { bs[c] = c < b ? 0.f : 1.f; bj[c] = 1000 + c; }
            merge8<KC>(ls, lj, bs, bj);
            const int zeros = std::min(KC, a + b);
            for (int p = 0; p < KC; ++p)
                CHECK(ls[p] == (p < zeros ? 0.f : 1.f), "merge8<%d> 0-1 a=%d b=%d p=%d", KC, a, b, p);
            for (int p = 0; p < KC; ++p) {
                const int id = lj[p];
                const float v = id >= 1000 ? (id - 1000 < b ? 0.f : 1.f) : (id < a ? 0.f : 1.f);
                CHECK(v == ls[p], "merge8<%d> id a=%d b=%d", KC, a, b);
            }
        }
}

template <int KC>
static void test_merge_random(std::mt19937 &g) {
    std::uniform_int_distribution<int> small(0, 12), len(0, KC);
    for (int t = 0; t < 20000; ++t) {
        // scores from a small set (many ties), +inf padding at the tails
        const int na = len(g), nb = small(g) % 9;
        std::vector<std::pair<float, int>> A, B;
        for (int p = 0; p < na; ++p) A.push_back({float(small(g)) - 3.f, p});
        for (int c = 0; c < nb; ++c) B.push_back({float(small(g)) - 3.f, 1000 + c});
        std::stable_sort(A.begin(), A.end(), [](auto x, auto y) { return x.first < y.first; });
        float ls[KC]; int lj[KC]; float bs[8]; int bj[8];
        for (int p = 0; p < KC; ++p) {
            ls[p] = p < na ? A[p].first : INFINITY;
            lj[p] = p < na ? A[p].second : -1;
        }
        for (int c = 0; c < 8; ++c) {
            bs[c] = c < nb ? B[c].first : INFINITY;
            bj[c] = c < nb ? B[c].second : -1;
        }
        sort8(bs, bj);
        std::vector<std::pair<float, int>> all;
        for (int p = 0; p < KC; ++p) all.push_back({ls[p], lj[p]});
        for (int c = 0; c < 8; ++c) all.push_back({bs[c], bj[c]});
        std::vector<float> want;
        for (auto &x : all) want.push_back(x.first);
        std::sort(want.begin(), want.end());
        merge8<KC>(ls, lj, bs, bj);
        for (int p = 0; p < KC; ++p) CHECK(ls[p] == want[p], "merge8<%d> random t=%d p=%d", KC, t, p);
        // each output pair is an input pair, none used twice (ids >= 0)
        std::vector<int> used;
        for (int p = 0; p < KC; ++p) {
            bool found = false;
            for (auto &x : all)
                if (x.second == lj[p] && x.first == ls[p]) { found = true; break; }
            CHECK(found, "merge8<%d> pair t=%d p=%d", KC, t, p);
            if (lj[p] >= 0) used.push_back(lj[p]);
        }
        std::sort(used.begin(), used.end());
        CHECK(std::adjacent_find(used.begin(), used.end()) == used.end(), "merge8<%d> dup id", KC);
    }
}

int main() {
    std::mt19937 g(12345);
    test_sort8();
    test_merge01<32>(); test_merge01<48>(); test_merge01<64>();
    test_merge_random<32>(g); test_merge_random<48>(g); test_merge_random<64>(g);
    std::printf("fails=%d\n", fails);
    return fails ? 1 : 0;
}
"""


def test_topk_networks(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "topk_harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "topk_harness"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails=0" in r.stdout
