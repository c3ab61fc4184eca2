"""FAMST build throughput on GB300.

Default workload: 1,000,000 unit vectors in 128-D drawn from a 1,000-cluster
mixture (k = 32, lambda = 10). A step is one full FAMST build (kNN graph,
components, connect, refine, MST, FP64 weight) of one cloud that is already
resident in HBM. Timing: W warm-up builds, then K builds between CUDA events
on the library's stream, bracketed by barrier + synchronize; max over ranks.
The cloud (512 MB) is larger than L2, so no flush is needed between steps.

Under torchrun each rank builds its own cloud (seed + rank): independent
problems, weak scaling, no data-path collective.

``--impl reference`` times the CPU oracle (the only implementation of the
method besides this one) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "points/sec for full FAMST build"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}
SMS = 152


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        p["_source"] = "measured"
        return p
    except Exception:
        p = dict(FALLBACK)
        p["_source"] = "fallback"
        return p


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_workload(w, rank: int):
    """Each rank builds its own independent cloud of the same recipe
    (seed + rank): weak scaling with no data-path exchange."""
    return workloads.Workload(w.name, w.n, w.d, w.k, w.lam, w.seed + rank, w.kind)


def max_over_ranks(x: float, pg, device) -> float:
    """The slowest rank's time (all_reduce MAX); identity without a group."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def throughput(world: int, n: int, steps: int, seconds: float) -> float:
    """Whole-job points per second: every rank builds `steps` clouds of n."""
    return world * n * steps / seconds


def source_hash(fname: str) -> str:
    p = os.path.join(ROOT, "paper_2507_14261_gb300", "csrc", fname)
    try:
        with open(p, "rb") as fh:
            return hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return ""


def traffic_from_profile(kernel: str, units: float):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.json: bytes per unit of work, measured on a smaller
    case of the same recipe), if it was taken on the current kernel source;
    else None. Units: candidate distances for the refinement kernel, visited
    (query, key) pairs for the distance tiles."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    for r in rec.get("entries", []):
        if r.get("kernel") == kernel and r.get("source_sha") == source_hash(r.get("source", "")):
            per_unit = r.get("dram_bytes_per_unit")
            if per_unit is not None:
                return float(per_unit) * units
    return None


def _oracle_knn_rate(X, k: int, threads: int, budget_s: float):
    import oracle
    n = X.shape[0]
    probe = 4 * threads
    oracle.knn(X, k, rows=(0, threads), threads=threads)  # warm the threads and caches
    t0 = time.perf_counter()
    oracle.knn(X, k, rows=(0, probe), threads=threads)
    dt = time.perf_counter() - t0
    S = int(max(probe, min(n, probe * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.knn(X, k, rows=(0, S), threads=threads)
    dt = time.perf_counter() - t0
    return S, dt


def cpu_baseline(X, k: int, budget_s: float = 15.0):
    """The oracle's brute-force kNN (Phase 1, the dominant cost of the
    oracle's build) on the first S query rows of the cloud, S sized to the
    time budget, on all host cores and on one thread; returns points/s and
    the sample description."""
    import oracle
    oracle.build()
    n = X.shape[0]
    cores = os.cpu_count() or 1
    S, dt = _oracle_knn_rate(X, k, cores, budget_s)
    S1, dt1 = _oracle_knn_rate(X, k, 1, budget_s / 3)
    return {"value": S / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle brute-force exact kNN of query rows 0..{S - 1} against all {n} "
                      f"points (Phase 1; the oracle's later phases cost <1% of it and are not "
                      f"timed); {dt:.1f} s",
            "single_thread": {"value": S1 / dt1, "unit": "points/s", "cores": 1,
                              "sample": f"query rows 0..{S1 - 1}; {dt1:.1f} s"},
            "cpu_model": _cpu_model()}


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def l2_copy_peak(device) -> dict:
    """Measured L2 bandwidth: a plain copy between two 16 MB buffers (both
    resident in the 129 MB L2), 64 copies per CUDA-graph replay so launch
    gaps do not count, read + write bytes over CUDA-event time, best of 10
    replays. The denominator for kernels that gather from L2."""
    import torch
    n = (16 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device=device)
    b = torch.empty_like(a)
    reps = 64
    s = torch.cuda.Stream(device)
    with torch.cuda.stream(s):
        for _ in range(3):
            b.copy_(a)
    torch.cuda.synchronize(device)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(reps):
            b.copy_(a)
    with torch.cuda.stream(s):
        g.replay()
    torch.cuda.synchronize(device)
    best = None
    for _ in range(10):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):   # replay() launches on the current stream
            e0.record(s)
            g.replay()
            e1.record(s)
        torch.cuda.synchronize(device)
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    gbs = 2.0 * a.numel() * 4 * reps / (best / 1e3) / 1e9
    del g
    return {"l2_gbs": gbs, "how": "torch copy 16 MB -> 16 MB, 64 per graph replay, best of 10"}


def fp32_simt_peak(device) -> dict:
    """Measured FP32 throughput without tensor cores: a 4096^3 FP32 matrix
    product with TF32 disabled (cuBLAS SGEMM on the FMA pipes), best of 5
    after a warm-up. The denominator for the FP32 distance tiles."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        m = 4096
        a = torch.randn(m, m, device=device)
        b = torch.randn(m, m, device=device)
        c = a @ b
        torch.cuda.synchronize(device)
        best = None
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize(device)
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return {"fp32_tflops": 2.0 * m ** 3 / (best / 1e3) / 1e12,
            "how": "torch FP32 matmul 4096^3, TF32 off, best of 5"}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = workloads.get(args.workload)
    X = w.points()
    cores = os.cpu_count() or 1
    # rows per step sized so that the whole run stays within a few minutes
    probe = 4 * cores
    oracle.knn(X, w.k, rows=(0, cores), threads=cores)  # warm the threads and caches
    t0 = time.perf_counter()
    oracle.knn(X, w.k, rows=(0, probe), threads=cores)
    per_row = (time.perf_counter() - t0) / probe
    S = int(max(probe, min(w.n, 10.0 / max(per_row, 1e-9))))
    times = []
    for s in range(args.warmup + args.steps):
        r0 = (s * S) % max(1, w.n - S)
        t0 = time.perf_counter()
        oracle.knn(X, w.k, rows=(r0, r0 + S), threads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = S * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "d": w.d, "k": w.k, "lambda": w.lam,
                   "sample_rows_per_step": S},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: oracle exact kNN of {S} query rows against all "
                                   f"{w.n} points (Phase 1)"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _knn_ms(c, X, k, prec, torch, reps=3):
    c.knn_graph(X, k, prec)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        nbr, dist = c.knn_graph(X, k, prec)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), nbr, dist


def precision_compare(fam, torch, bf16_peak=None) -> dict:
    """Phase 1 of the 100k x 128 mixture (k = 16) by brute force in every
    tile precision: tcgen05 BF16 hi/lo, BF16, E4M3 (kind::f8f6f4) and the
    FP32 SIMT tiles, median of 3 after a warm-up. All return the exact kNN
    graph (compared here); the precisions differ in tile time and in how
    many rows their error bound leaves to the FP32 recomputation (read from
    one build's statistics)."""
    w = workloads.get("blobs_100k")
    X = torch.from_numpy(w.points()).cuda()
    c = fam.Context(torch.cuda.current_device())
    c.set_knn_pruning(False)
    out = {"workload": "blobs_100k (100k x 128, k = 16), kNN stage, no tile pruning"}
    graphs = {}
    for prec in ("bf16x3", "bf16", "fp8", "fp32"):
        ms, nbr, dist = _knn_ms(c, X, w.k, prec, torch)
        graphs[prec] = (nbr, dist)
        _, info = c.build(X, w.k, w.lam, 1, prec)
        out[prec] = {"ms": ms, "points_per_s": w.n / (ms / 1e3),
                     "uncertified_rows": info.uncertified_rows,
                     "ms_tiles": info.ms_knn_tiles, "ms_rerank": info.ms_rerank}
        if prec != "fp32" and bf16_peak:
            kel = 128 if prec == "fp8" else 64
            d_pad = -(-w.d // kel) * kel
            nt = -(-w.n // 128)
            # every tile pair of the padded square; 2 d_pad FLOP per pair
            # (BF16 hi/lo issues three products: 'issued_frac')
            flops = 2.0 * (nt * 128) ** 2 * d_pad
            peak = bf16_peak * (2.0 if prec == "fp8" else 1.0)
            out[prec]["tiles_tflops"] = flops / (info.ms_knn_tiles / 1e3) / 1e12
            out[prec]["tiles_frac"] = out[prec]["tiles_tflops"] / peak
            out[prec]["issued_frac"] = out[prec]["tiles_frac"] * (3 if prec == "bf16x3" else 1)
            out[prec]["tiles_peak"] = ("measured bf16 x 2 (nominal fp8:bf16 ratio)"
                                       if prec == "fp8" else "measured bf16")
    # FP32 SIMT tiles: 2 d FLOP per (query, key) pair over the whole stage
    # (FP32 tiles, candidate re-rank), against a measured SGEMM rate
    f32pk = fp32_simt_peak(X.device)
    fl32 = 2.0 * w.n * w.n * w.d / (out["fp32"]["ms"] / 1e3) / 1e12
    out["fp32"].update({"stage_tflops": fl32, "peak_fp32_tflops": f32pk["fp32_tflops"],
                        "frac": fl32 / f32pk["fp32_tflops"], "peak_how": f32pk["how"]})
    ref = graphs["fp32"]
    out["identical_graphs"] = bool(all(torch.equal(g[0], ref[0]) and torch.equal(g[1], ref[1])
                                       for g in graphs.values()))
    out["recall_at_k"] = 1.0 if out["identical_graphs"] else None
    out["speedup_bf16x3_over_fp32"] = out["fp32"]["ms"] / out["bf16x3"]["ms"]
    out["speedup_fp8_over_bf16x3"] = out["bf16x3"]["ms"] / out["fp8"]["ms"]
    c.close()
    return out


def fp8_on_workload(fam, torch, X, w, prec, tree_ref) -> dict:
    """One build of the timed workload with E4M3 tiles (no tile pruning)
    after a warm-up, against the timed precision's tree: the same tree, its
    kNN-stage time and the rows its error bound could not certify."""
    c = fam.Context(torch.cuda.current_device())
    c.build(X, w.k, w.lam, 1, "fp8")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree, info = c.build(X, w.k, w.lam, 1, "fp8")
    torch.cuda.synchronize()
    out = {"ms_build": 1e3 * (time.perf_counter() - t0), "ms_knn": info.ms_knn,
           "ms_tiles": info.ms_knn_tiles, "uncertified_rows": info.uncertified_rows,
           "uncertified_frac": info.uncertified_rows / w.n,
           "same_tree_as": prec,
           "same_tree": bool(torch.equal(tree.u, tree_ref.u) and torch.equal(tree.v, tree_ref.v)
                             and torch.equal(tree.w, tree_ref.w)),
           "timing": "one build after a warm-up, host wall clock; stage times by CUDA events"}
    c.close()
    return out


def nndescent_sub(fam, torch, X, w, prec, quality, S=None, iters=10, delta=0.001) -> dict:
    """NN-Descent as Phase 1 on the timed cloud: famst_knn_nndescent timed
    by CUDA events after a warm-up, recall@k against the exact tiles'
    graph, join pairs per iteration, and one build with it as Phase 1."""
    c = fam.Context(torch.cuda.current_device())
    S = min(w.k, 32) if S is None else S
    exact_nbr, _ = c.knn_graph(X, w.k, prec)
    c.knn_nndescent(X, w.k, S, iters, delta, 1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    nbr, dist, it, upd, prs = c.knn_nndescent(X, w.k, S, iters, delta, 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    hit = 0
    for r0 in range(0, w.n, 65536):   # recall@k in slices (bounded memory)
        a, b = nbr[r0:r0 + 65536], exact_nbr[r0:r0 + 65536]
        hit += int((a.unsqueeze(2) == b.unsqueeze(1)).any(2).sum().item())
    out = {"S": S, "max_iters": iters, "delta": delta, "ms": ms, "iters": it,
           "updates": upd.tolist(), "join_pairs": prs.tolist(),
           "recall_at_k": hit / (w.n * w.k),
           "points_per_s": w.n / (ms / 1e3),
           "timing": "CUDA events around famst_knn_nndescent after a warm-up"}
    c.set_knn_method("nndescent", S, iters, delta)
    tree, info = c.build(X, w.k, w.lam, 1, prec)
    out["build"] = {"W": tree.W, "ms_knn": info.ms_knn, "ms_total": info.ms_total,
                    "t": info.t, "refine_sweeps": info.refine_sweeps,
                    "knn_iters": info.knn_iters}
    if quality is not None and quality["W_exact"] > 0:
        out["build"]["rel_err"] = (tree.W - quality["W_exact"]) / quality["W_exact"]
        out["build"]["rel_err_exact_knn"] = quality["rel_err"]
    c.close()
    return out


def batch_sub(fam, torch, local: int, prec: str, steps: int = 5) -> dict:
    clouds = workloads.batch_clouds()
    off = np.zeros(len(clouds) + 1, np.int64)
    for b, cl in enumerate(clouds):
        off[b + 1] = off[b] + cl.shape[0]
    dims = np.array([cl.shape[1] for cl in clouds], np.int32)
    X = torch.from_numpy(np.concatenate([cl.ravel() for cl in clouds]).astype(np.float32)).cuda()
    c = fam.Context(local)
    k, lam = 16, 5
    for _ in range(3):
        c.build_batched(X, off, dims, k, lam, 1, prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        _, _, _, info = c.build_batched(X, off, dims, k, lam, 1, prec)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    c.close()
    return {"points_per_s": int(off[-1]) * steps / dt, "ms_per_step": 1e3 * dt / steps,
            "clouds": len(clouds), "points": int(off[-1]), "steps": steps,
            "graph_replayed": info.graph_replayed, "graph_kernels": info.graph_kernels,
            "tensor_clouds": info.tensor_clouds, "uncertified_rows": info.uncertified_rows,
            "tile_shape": {"epilogue_warps": info.tile_epilogue_warps,
                           "ring_stages": info.tile_stages},
            "timing": "host wall clock around synchronised replays"}


def run_sweep(args, world, rank, local):
    """The shape of the paper's k / lambda study (Sec. 5: relative error and
    time against k and lambda) on the synthetic stand-ins for its data: the
    2,000 x 16 and 100,000 x 128 Gaussian mixtures. For every (k, lambda) one
    JSON line: build time (median of 3 after a warm-up, CUDA events),
    W, Eq. 1's relative error against the exact EMST of the same cloud (GPU
    Boruvka over exact masked 1-NN passes; at 2,000 points also checked
    against the oracle's Prim), t, |E| and the refinement sweeps."""
    import torch
    import paper_2507_14261_gb300 as fam
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    ctx = fam.Context(local)
    ks = [int(x) for x in args.sweep_k.split(",")]
    lams = [int(x) for x in args.sweep_lambda.split(",")]
    for name in args.sweep_workloads.split(","):
        w = workloads.get(name)
        X_np = w.points()
        X = torch.from_numpy(X_np).cuda()
        T, _ = ctx.emst_exact(X, args.prec)
        W_exact = T.W
        prim = None
        if w.n <= 5000:
            import oracle
            oracle.build()
            prim = oracle.prim_exact(X_np).W
        for k in ks:
            for lam in lams:
                if k > w.n - 1:
                    continue
                ctx.build(X, k, lam, 1, args.prec)
                ts, info = [], None
                for _ in range(3):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    tree, info = ctx.build(X, k, lam, 1, args.prec)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = statistics.median(ts)
                line = {"sweep": "k_lambda", "workload": name, "n": w.n, "d": w.d, "k": k,
                        "lambda": lam, "prec": args.prec, "ms": ms,
                        "points_per_s": w.n / (ms / 1e3), "W": tree.W, "W_exact": W_exact,
                        "rel_err": (tree.W - W_exact) / W_exact, "t": info.t, "m": info.m,
                        "refine_sweeps": info.refine_sweeps,
                        "ms_stages": {"knn": info.ms_knn, "connect": info.ms_connect,
                                      "refine": info.ms_refine, "mst": info.ms_mst}}
                if prim is not None:
                    line["W_exact_oracle_prim"] = prim
                print(json.dumps(line), flush=True)
    return 0


def run_batch(args, world, rank, local):
    """256 clouds (n_b ~ U{500..20000}, d_b in {3, 32, 128}, 5-20 clusters,
    k=16, lambda=5) per step through famst_build_batched: one captured CUDA
    graph replay per step. Each rank builds its own batch (seed offset)."""
    import torch
    import paper_2507_14261_gb300 as fam
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    clouds = workloads.batch_clouds(base_seed=1000 + 100000 * rank)
    off = np.zeros(len(clouds) + 1, np.int64)
    for b, c in enumerate(clouds):
        off[b + 1] = off[b] + c.shape[0]
    dims = np.array([c.shape[1] for c in clouds], np.int32)
    flat = np.concatenate([c.ravel() for c in clouds]).astype(np.float32)
    X = torch.from_numpy(flat).cuda()
    N = int(off[-1])
    ctx = fam.Context(local)
    k, lam = 16, 5
    for _ in range(args.warmup):
        trees, W, t, info = ctx.build_batched(X, off, dims, k, lam, 1, args.prec)
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launches
    t0 = time.perf_counter()
    for _ in range(args.steps):
        trees, W, t, info = ctx.build_batched(X, off, dims, k, lam, 1, args.prec)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
    clocks = sampler.stop()
    launches = ctx.launches - launches0
    # algorithmic work of the distance tiles: 2 n_b^2 d_b per cloud
    flops = float(sum(2.0 * (off[b + 1] - off[b]) ** 2 * dims[b] for b in range(len(clouds))))
    pk = peaks()
    achieved = flops * args.steps / dt / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": throughput(world, N, args.steps, dt), "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if args.prec != "fp32" else "f32",
            "data": "synthetic (seeded; 256 clouds, inputs larger than L2)",
            "config": {"workload": "batch_256", "clouds": len(clouds), "points": N, "k": k,
                       "lambda": lam, "prec": args.prec, "parallelism": f"replicas x{world}",
                       "graph": "one captured CUDA graph replay per step"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops"], "traffic": None,
                         "kernel": "whole batched build (distance FLOPs / step time; a lower bound "
                                   "on the distance kernel's own rate)"},
            "cpu_baseline": None, "e2e": None, "clocks": clocks, "gpu_launches": launches,
            "build": {"tile_epilogue_warps": info.tile_epilogue_warps, "tile_stages": info.tile_stages,
                  "tensor_clouds": info.tensor_clouds, "uncertified_rows": info.uncertified_rows,
                      "m": info.m, "refine_sweeps": info.refine_sweeps,
                      "graph_kernels": info.graph_kernels, "graph_replayed": info.graph_replayed},
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="famst", choices=["famst", "reference"])
    ap.add_argument("--workload", default="sphere_1m")
    ap.add_argument("--n", type=int, default=None,
                    help="same recipe at another size (profiling runs); default: the workload's n")
    ap.add_argument("--prec", default=os.environ.get("FAMST_BENCH_PREC", "bf16x3"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the exact EMST (Eq. 1 relative error, after the timed region)")
    ap.add_argument("--sweep", action="store_true",
                    help="k / lambda study on the 2k x 16 and 100k x 128 mixtures (JSON lines)")
    ap.add_argument("--sweep-k", default="5,10,16,20,32")
    ap.add_argument("--sweep-lambda", default="1,2,5,10")
    ap.add_argument("--sweep-workloads", default="blobs_small,blobs_100k")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision comparison and the batch_256 sub-object")
    ap.add_argument("--knn", default="exact", choices=["exact", "nndescent"],
                    help="Phase 1 of the timed builds: the exact tiles (default) or NN-Descent "
                         "(S = min(k, 32), at most 10 iterations, delta 0.001)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    import torch
    import paper_2507_14261_gb300 as fam

    if args.workload == "batch_256":
        return run_batch(args, world, rank, local)
    if args.sweep:
        return run_sweep(args, world, rank, local)
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    w = workloads.get(args.workload)
    if args.n is not None:
        w = workloads.Workload(w.name, args.n, w.d, w.k, w.lam, w.seed, w.kind)
    X_np = rank_workload(w, rank).points()
    X = torch.from_numpy(X_np).cuda()
    ctx = fam.Context(local)
    if args.knn == "nndescent":
        ctx.set_knn_method("nndescent", min(w.k, 32), 10, 0.001)
    stream = torch.cuda.current_stream()

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    infos = []
    for _ in range(args.warmup):
        tree, info = ctx.build(X, w.k, w.lam, 1, args.prec)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        tree, info = ctx.build(X, w.k, w.lam, 1, args.prec)
        infos.append(info.as_dict())
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    launches = ctx.launches - launches0
    ms = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
    value = throughput(world, w.n, args.steps, ms / 1e3)

    # end to end through the host-buffer entry point: pinned X in, tree out
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X_np).pin_memory()
        out = (torch.empty(w.n - 1, dtype=torch.int32).pin_memory(),
               torch.empty(w.n - 1, dtype=torch.int32).pin_memory(),
               torch.empty(w.n - 1, dtype=torch.float32).pin_memory())
        for _ in range(args.warmup):   # the same warm-up as the device-timed builds
            ctx.build_host(Xh, w.k, w.lam, 1, args.prec, out=out)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.build_host(Xh, w.k, w.lam, 1, args.prec, out=out)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
        e2e = {"value": throughput(world, w.n, args.steps, dt), "unit": "points/s",
               "h2d_bytes_per_step": int(X_np.nbytes),
               "d2h_bytes_per_step": int((w.n - 1) * 12 + 8)}

    # Rooflines per kernel, each from that kernel's own CUDA-event time on
    # the library's stream during the timed builds (famst_build_info).
    pk = peaks()
    l2 = l2_copy_peak(X.device)
    mean = lambda key: statistics.mean(i[key] for i in infos)  # noqa: E731
    ms_tiles, ms_rerank = mean("ms_knn_tiles"), mean("ms_rerank")
    ms_refk, ms_conk = mean("ms_refine_kernel"), mean("ms_connect_kernel")
    frac_tiles = mean("knn_tile_fraction")
    evals, canon = mean("refine_distance_evals"), mean("refine_canonical_evals")
    nq, nk = (w.n + 127) // 128, (w.n + 255) // 256
    kernels = {}
    if args.prec != "fp32" and ms_tiles > 0:
        # 2 d FLOP per (query, key) pair of every visited tile pair; BF16x3
        # issues three products per pair, its own tensor ceiling is 1/3
        pairs = nq * nk * 128 * 256 * frac_tiles
        ach = 2.0 * w.d * pairs / (ms_tiles / 1e3) / 1e12
        prods = 3 if args.prec == "bf16x3" else 1
        kernels["knn_tiles"] = {
            "bound": "tensor", "ms": ms_tiles, "achieved": ach, "peak": pk["bf16_tflops"],
            "unit": "TFLOP/s", "frac": ach / pk["bf16_tflops"],
            "frac_of_x3_ceiling": ach * prods / pk["bf16_tflops"],
            "tile_fraction": frac_tiles, "kernel": "knn_tc_kernel",
            "note": "visited tile pairs' 2 d FLOP per pair over the tile kernel's own time; "
                    "peak = measured BF16 burst"}
    kernels["knn_stage"] = {"ms": mean("ms_knn"),
                            "note": "whole Phase 1: operand prep, pruning partition, tiles, "
                                    "re-rank, fallback rows"}
    if ms_rerank > 0:
        # per query row: (KC - 1) candidate FP32 rows gathered (KC = 48 for k = 32)
        kc = 32 if w.k <= 21 else (48 if w.k <= 37 else 64)
        rb = w.n * (kc - 1) * w.d * 4.0 + w.n * w.k * 8.0
        kernels["rerank"] = {"bound": "l2", "ms": ms_rerank,
                             "achieved": rb / (ms_rerank / 1e3) / 1e9, "peak": l2["l2_gbs"],
                             "unit": "GB/s", "frac": rb / (ms_rerank / 1e3) / 1e9 / l2["l2_gbs"],
                             "kernel": "rerank_sorted_kernel",
                             "note": "(KC - 1) FP32 candidate rows per query + nbr/dist out"}
    if ms_refk > 0:
        # bytes Algorithm 4's kernels read: every staged candidate BF16 row
        # (2 ld B) with its list entry (id, eb, ||h||^2: 12 B), every fixed
        # point's BF16 row with its scan record (2 ld + 24 B), and two FP32 rows
        # per canonical evaluation (2 x 4 d B)
        ld = (w.d + 63) // 64 * 64
        staged, fixed = mean("refine_rows_staged"), mean("refine_fixed_rows")
        rbytes = staged * (2.0 * ld + 12.0) + fixed * (2.0 * ld + 24.0) + canon * 8.0 * w.d
        ach = rbytes / (ms_refk / 1e3) / 1e9
        kernels["refine"] = {
            "bound": "l2", "ms": ms_refk, "achieved": ach, "peak": l2["l2_gbs"], "unit": "GB/s",
            "frac": ach / l2["l2_gbs"], "distance_evals": evals, "canonical_evals": canon,
            "rows_staged": staged, "fixed_rows": fixed,
            "pairs_per_s": evals / (ms_refk / 1e3),
            "kernel": "refine_group_kernel + refine_staged_kernel",
            "note": "bytes the kernels read (staged candidate rows once per scanned vertex and "
                    "round, fixed rows, canonical survivors' FP32 rows) over the kernels' own "
                    "time, against the measured L2 copy bandwidth; the kernels are latency "
                    "bound (see profiles/), so the fraction is well below 1"}
    if ms_conk > 0:
        m_e = infos[-1]["m"]
        draws = m_e / w.lam * (w.lam * w.lam)
        if infos[-1]["refine_filter"] == 2:
            # builds holding the centred BF16 rows filter on those: per draw
            # two rows of ld BF16 values plus their norm and error bound
            ld = -(-w.d // 64) * 64
            cb = draws * 2.0 * (2.0 * ld + 8.0)
            kname = "connect_half_kernel"
            note = ("lambda^2 draws x two BF16 rows (+ norm, error bound) per component pair; "
                    "the canonical survivors' FP32 rows are not counted")
        else:
            cb = draws * 2.0 * w.d * 4.0
            kname = "connect_filtered_kernel"
            note = "lambda^2 draws x two FP32 rows per component pair"
        kernels["connect"] = {"bound": "l2", "ms": ms_conk,
                              "achieved": cb / (ms_conk / 1e3) / 1e9, "peak": l2["l2_gbs"],
                              "unit": "GB/s", "frac": cb / (ms_conk / 1e3) / 1e9 / l2["l2_gbs"],
                              "kernel": kname, "note": note}
    # dW/dX of the tree weight (the tree held fixed), after the timed builds:
    # per vertex its own row, its tree neighbours' rows and its gradient row
    # ((n - 1) d 4 B x 4 algorithmic bytes), timed on the library's stream
    gx = torch.empty_like(X)
    ctx.mst_backward(X, tree.u, tree.v, 1.0, out=gx)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    b0.record(stream)
    for _ in range(reps):
        ctx.mst_backward(X, tree.u, tree.v, 1.0, out=gx)
    b1.record(stream)
    torch.cuda.synchronize()
    ms_bwd = b0.elapsed_time(b1) / reps
    bwd_bytes = (w.n - 1) * w.d * 4 * 4
    kernels["backward"] = {"bound": "hbm", "ms": ms_bwd,
                           "achieved": bwd_bytes / (ms_bwd / 1e3) / 1e9,
                           "peak": pk["hbm_gbs"], "unit": "GB/s",
                           "frac": bwd_bytes / (ms_bwd / 1e3) / 1e9 / pk["hbm_gbs"],
                           "kernel": "famst_mst_backward (edge lengths, incidence sort, per-vertex sums)"}
    del gx
    # the dominant kernel of the build by its own time
    cands = {kk: v for kk, v in kernels.items() if "bound" in v and kk != "backward"}
    dom = max(cands, key=lambda kk: cands[kk]["ms"])
    kd = kernels[dom]
    units = evals if dom == "refine" else frac_tiles * nq * nk * 128 * 256
    traffic = traffic_from_profile("refine_group_kernel" if dom == "refine" else kd["kernel"],
                                   units)
    roofline = {"bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
                "unit": kd["unit"], "frac": kd["frac"], "traffic": traffic,
                "kernel": kd["kernel"], "ms_per_launch": kd["ms"],
                "peak_source": ("measured in this run: " + l2["how"]) if kd["bound"] == "l2"
                else "MEASURED_PEAKS.json (" + pk["_source"] + ")"}

    # Eq. 1: relative error of the FAMST tree against the exact EMST, both
    # on the GPU, outside the timed region
    quality = None
    if not args.no_quality:
        t0 = time.perf_counter()
        T, rounds = ctx.emst_exact(X, args.prec)
        torch.cuda.synchronize()
        quality = {"W_famst": tree.W, "W_exact": T.W,
                   "rel_err": (tree.W - T.W) / T.W if T.W > 0 else 0.0,
                   "exact": "GPU Boruvka over masked exact 1-NN passes",
                   "emst_rounds": rounds, "emst_s": time.perf_counter() - t0}

    # Like-for-like precision comparison on the 100k x 128 mixture (k = 16):
    # Phase 1 brute force (no tile pruning) with BF16 hi/lo tensor tiles
    # against the FP32 SIMT tiles; both return the exact kNN graph (recall@k
    # = 1.0, checked equal here), so only the distance arithmetic differs.
    precision = fp8 = None
    if not args.no_extras and rank == 0:
        precision = precision_compare(fam, torch, pk.get("bf16_tflops"))
        fp8 = fp8_on_workload(fam, torch, X, w, args.prec, tree)

    # 256 clouds through the batched entry point (one CUDA-graph replay per
    # step), after the timed region
    batch = None
    if not args.no_extras and rank == 0:
        batch = batch_sub(fam, torch, local, args.prec)

    # The nearest-pair connect (the lambda nearest cross pairs of every
    # component pair instead of Algorithm 3's samples) on the same cloud,
    # once, after the timed region: W and Eq. 1's error against Algorithm 3's
    nearest = None
    if not args.no_extras and rank == 0:
        c2 = fam.Context(local)
        c2.set_connect_mode("nearest")
        tree_n, info_n = c2.build(X, w.k, w.lam, 1, args.prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tree_n, info_n = c2.build(X, w.k, w.lam, 1, args.prec)
        torch.cuda.synchronize()
        nearest = {"W": tree_n.W, "W_random_alg3": tree.W,
                   "ms_build": 1e3 * (time.perf_counter() - t0), "ms_connect": info_n.ms_connect,
                   "ms_refine": info_n.ms_refine, "refine_sweeps": info_n.refine_sweeps,
                   "timing": "one build after a warm-up, host wall clock"}
        if quality is not None and quality["W_exact"] > 0:
            nearest["rel_err"] = (tree_n.W - quality["W_exact"]) / quality["W_exact"]
            nearest["rel_err_random_alg3"] = quality["rel_err"]
        c2.close()

    # Phase 1 by NN-Descent (the paper's own Phase 1 method) on the same
    # cloud, after the timed region: its time, iterations and recall@k
    # against the exact graph, and a whole build on it (W, Eq. 1's error)
    nndescent = None
    if not args.no_extras and rank == 0:
        nndescent = nndescent_sub(fam, torch, X, w, args.prec, quality)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(X_np, w.k)

    last = infos[-1]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec == "fp32" else "bf16",
            "data": "synthetic (seeded; inputs larger than L2, no flush)",
            "config": {"workload": w.name, "n": w.n, "d": w.d, "k": w.k, "lambda": w.lam,
                       "prec": args.prec, "knn": args.knn,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (X = %d MB)" % (X_np.nbytes >> 20)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "quality": quality, "kernels": kernels,
            "l2_peak": l2, "precision_compare": precision, "batch_256": batch,
            "connect_nearest": nearest, "fp8_tiles": fp8, "nndescent": nndescent,
            "stages_ms": {k2: last[k2] for k2 in ("ms_knn", "ms_components", "ms_connect",
                                                  "ms_refine", "ms_mst", "ms_total")},
            "build": {"t": last["t"], "m": last["m"], "refine_sweeps": last["refine_sweeps"],
                      "boruvka_rounds": last["boruvka_rounds"], "W": last["W"],
                      "W64": last["W64"], "uncertified_rows": last["uncertified_rows"],
                      "knn_tile_fraction": last["knn_tile_fraction"],
                      "refine_distance_evals": last["refine_distance_evals"],
                      "refine_canonical_evals": last["refine_canonical_evals"],
                      "refine_filter": last["refine_filter"],
                      "knn_iters": last["knn_iters"]},
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
