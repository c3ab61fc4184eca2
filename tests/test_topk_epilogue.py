"""The tile kernel's per-row top-KC algorithm, emulated on the host with the
kernel's own networks (csrc/topk_merge.cuh), against brute force (CPU).

Phase 1 (Algorithm 1, GetANNs) keeps for every query row the KC smallest
scores s(i, j) among its keys, starting below a threshold thr0, and reports
KC - 1 candidates with s+ = min(KC-th score, thr0). In the kernel two warps
share a row, each on half of a tile's columns: each stages the columns below
its threshold, merges them into its own list eight at a time whenever a
stage may overflow (the warp flushes when any lane's stage is nearly full,
so a row flushes at times set by other rows), filters with the smaller of
its own and its partner's KC-th score, and at the end the second list is
merged into the first. A long key list may also be split into parts whose
rows are recombined afterwards.

The emulation keeps that structure per row (chunks of 16 columns, stage of
24, flush when more than 8 are staged or at random extra times) and checks
that the reported candidate scores and s+ equal brute force for random
scores with ties, +inf keys (masked), start thresholds, KC = 32, 48, 64,
whole or split lists.
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2507_14261_gb300", "csrc")

HARNESS = r"""
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "topk_merge.cuh"
using namespace famst::topk;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails < 10) { std::printf(__VA_ARGS__); std::printf("\n"); } ++fails; } } while (0)
static const float INF = INFINITY;

template <int KC> struct Half {
    float ls[KC]; int lj[KC];
    std::vector<std::pair<float, int>> stage;
    Half() { for (int p = 0; p < KC; ++p) { ls[p] = INF; lj[p] = -1; } }
    // merge the stage into the list, eight at a time, filtering with
    // min(own KC-th, partner's published KC-th)
    void flush(float partner) {
        for (size_t q0 = 0; q0 < stage.size(); q0 += 8) {
            const float lim = std::min(ls[KC - 1], partner);
            float bs[8]; int bj[8]; int nq = 0;
            for (int c = 0; c < 8; ++c) {
                bs[c] = INF; bj[c] = -1;
                if (q0 + c < stage.size() && stage[q0 + c].first < lim) {
                    bs[c] = stage[q0 + c].first; bj[c] = stage[q0 + c].second; ++nq;
                }
            }
            if (nq == 0) continue;
            sort8(bs, bj);
            merge8<KC>(ls, lj, bs, bj);
        }
        stage.clear();
    }
};

// one row over the keys [0, n) in 256-column tiles; returns the KC - 1
// reported (score, id) and s+
template <int KC>
static void row(const std::vector<float> &sc, int k0, int k1, float thr0, std::mt19937 &g,
                std::vector<std::pair<float, int>> &out, float &splus) {
    Half<KC> h[2];
    float pub[2] = {INF, INF};
    float thr[2] = {thr0, thr0};
    std::uniform_int_distribution<int> coin(0, 9);
    for (int t0 = k0; t0 < k1; t0 += 256) {
        for (int half = 0; half < 2; ++half) {
            thr[half] = std::min(thr[half], pub[1 - half]);
            for (int ch = 0; ch < 8; ++ch) {
                for (int c = 0; c < 16; ++c) {
                    const int j = t0 + half * 128 + ch * 16 + c;
                    if (j >= k1) break;
                    if (sc[j] < thr[half]) h[half].stage.push_back({sc[j], j});
                }
                // own overflow guard, or another lane of the warp forcing a flush
                if (h[half].stage.size() > 8 || coin(g) == 0) {
                    h[half].flush(pub[1 - half]);
                    pub[half] = h[half].ls[KC - 1];
                    thr[half] = std::min(std::min(h[half].ls[KC - 1], pub[1 - half]), thr0);
                }
            }
        }
    }
    for (int half = 0; half < 2; ++half) {
        h[half].flush(pub[1 - half]);
        pub[half] = h[half].ls[KC - 1];
    }
    // the second list into the first, in ascending batches of eight
    Half<KC> &a = h[0];
    for (int p0 = 0; p0 < KC; p0 += 8) {
        const float lim = a.ls[KC - 1];
        float bs[8]; int bj[8]; int nq = 0;
        for (int c = 0; c < 8; ++c) {
            const bool in = h[1].ls[p0 + c] < lim;
            bs[c] = in ? h[1].ls[p0 + c] : INF; bj[c] = in ? h[1].lj[p0 + c] : -1; nq += in;
        }
        if (nq == 0) break;
        merge8<KC>(a.ls, a.lj, bs, bj);
    }
    out.clear();
    for (int p = 0; p < KC - 1; ++p) out.push_back({a.ls[p], a.lj[p]});
    splus = std::min(a.ls[KC - 1], thr0);
}

template <int KC>
static void check(std::mt19937 &g, int t) {
    std::uniform_int_distribution<int> nd(1, 1500), tie(-6, 6);
    const int n = nd(g);
    std::vector<float> sc(n);
    const bool ties = t % 3 == 0;
    std::normal_distribution<float> nrm;
    for (int j = 0; j < n; ++j) sc[j] = ties ? float(tie(g)) : nrm(g);
    for (int j = 0; j < n; ++j) if (g() % 17 == 0) sc[j] = INF;   // masked keys
    std::vector<float> srt(sc);
    std::sort(srt.begin(), srt.end());
    float thr0 = INF;
    if (t % 4 != 0) thr0 = srt[g() % n];
    // brute force: the KC smallest scores below thr0
    std::vector<float> below;
    for (float s : srt) if (s < thr0) below.push_back(s);
    while ((int)below.size() < KC) below.push_back(INF);
    const float want_splus = std::min(below[KC - 1], thr0);
    // whole list, or split into parts merged by the rule
    const int P = (t % 2) ? 1 : 2 + int(g() % 4);
    std::vector<std::pair<float, int>> out, all;
    float splus = INF, sp_min = INF;
    for (int p = 0; p < P; ++p) {
        const int k0 = int(int64_t(n) * p / P), k1 = int(int64_t(n) * (p + 1) / P);
        std::vector<std::pair<float, int>> o; float s;
        row<KC>(sc, k0, k1, thr0, g, o, s);
        sp_min = std::min(sp_min, s);
        all.insert(all.end(), o.begin(), o.end());
    }
    std::sort(all.begin(), all.end());
    if (P == 1) { out.assign(all.begin(), all.begin() + (KC - 1)); splus = sp_min; }
    else {
        while ((int)all.size() < KC) all.push_back({INF, -1});
        out.assign(all.begin(), all.begin() + (KC - 1));
        splus = std::min(all[KC - 1].first, sp_min);
    }
    for (int p = 0; p < KC - 1; ++p) {
        CHECK(out[p].first == below[p], "KC=%d t=%d p=%d score %g want %g", KC, t, p, out[p].first, below[p]);
        if (out[p].second >= 0) CHECK(sc[out[p].second] == out[p].first, "KC=%d t=%d id", KC, t);
    }
    CHECK(splus == want_splus, "KC=%d t=%d splus %g want %g", KC, t, splus, want_splus);
}

int main() {
    std::mt19937 g(2507);
    for (int t = 0; t < 1500; ++t) { check<32>(g, t); check<48>(g, t); check<64>(g, t); }
    std::printf("fails=%d\n", fails);
    return fails ? 1 : 0;
}
"""


def test_epilogue_lists_equal_brute_force(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "epilogue.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "epilogue"
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails=0" in r.stdout
