"""FAMST CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never does, and this
package never imports the library: the two share no code.

The arithmetic lives in ``famst_oracle.c`` (plain C, compiled on first use
with gcc, ``-O2 -ffp-contract=off``, OpenMP only to spread independent rows
over cores). This module only marshals numpy arrays and strings the stages
together in the order of Algorithm 1:

    kNN graph  ->  Components (Alg. 2)  ->  RandomEdges (Alg. 3)
    ->  repeat RefineEdges (Alg. 4) until |Delta| = 0  ->  Kruskal

Pins (checked by ``tests/test_oracle_*.py``): exact integer-coordinate
distances and correctly rounded sqrt; brute-force kNN against
``torch.cdist`` in float64; components against scipy's connected
components; Philox4x32-10 against the published known-answer vectors;
Kruskal and Prim against each other and against enumeration of all
spanning trees; closed forms (collinear points, unit grid, regular polygon);
k = n-1 reduces FAMST to the exact MST; a hand-worked 1-D refinement; the
gradient against central finite differences and a two-point closed form.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "famst_oracle.c")
_LIB = None
_LOCK = threading.Lock()

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def lib_path() -> str:
    return os.path.join(_HERE, "_build", f"libfamst_oracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle for this machine (host C, no CUDA)."""
    out = lib_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            c = ctypes
            L.or_dist32.argtypes = [_f32p, _f32p, c.c_int]
            L.or_dist32.restype = c.c_float
            L.or_dist64.argtypes = [_f32p, _f32p, c.c_int]
            L.or_dist64.restype = c.c_double
            L.or_knn.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, c.c_int64,
                                 c.c_int64, _i32p, _f32p, c.c_int]
            L.or_knn.restype = None
            L.or_build_graph.argtypes = [_i32p, c.c_int64, c.c_int, _i64p, _i32p]
            L.or_build_graph.restype = c.c_int64
            L.or_components.argtypes = [c.c_int64, _i64p, _i32p, _i32p, _i32p, _i64p]
            L.or_components.restype = c.c_int64
            L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.or_philox4x32_10.restype = None
            L.or_nndescent.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, c.c_int, c.c_int,
                                       c.c_double, c.c_uint64, c.c_void_p, _i32p, _f32p,
                                       _i64p, _i64p]
            L.or_nndescent.restype = c.c_int
            L.or_random_edges.argtypes = [_f32p, c.c_int, _i32p, _i64p, c.c_int64,
                                          c.c_int, c.c_uint64, _i32p, _i32p, _f32p,
                                          _i32p, _i32p]
            L.or_random_edges.restype = c.c_int64
            L.or_nearest_edges.argtypes = [_f32p, c.c_int, _i32p, _i64p, c.c_int64, c.c_int,
                                           _i32p, _i32p, _f32p, _i32p, _i32p]
            L.or_nearest_edges.restype = c.c_int64
            L.or_refine_sweep.argtypes = [_f32p, c.c_int, _i64p, _i32p, _i32p,
                                          c.c_int64, _i32p, _i32p, _f32p, _i32p,
                                          _i32p, _u8p]
            L.or_refine_sweep.restype = c.c_int64
            L.or_kruskal.argtypes = [c.c_int64, _i32p, _f32p, c.c_int, c.c_int64,
                                     _i32p, _i32p, _f32p, _i32p, _i32p, _f32p,
                                     ctypes.POINTER(c.c_double)]
            L.or_kruskal.restype = c.c_int64
            L.or_prim.argtypes = [_f32p, c.c_int64, c.c_int, _i32p, _i32p, _f32p,
                                  ctypes.POINTER(c.c_double), c.c_int]
            L.or_prim.restype = None
            L.or_tree_weight64.argtypes = [_f32p, c.c_int, _i32p, _i32p, c.c_int64]
            L.or_tree_weight64.restype = c.c_double
            L.or_mst_grad.argtypes = [_f32p, c.c_int64, c.c_int, _i32p, _i32p,
                                      c.c_int64, _f64p]
            L.or_mst_grad.restype = None
            _LIB = L
    return _LIB


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def threads_default() -> int:
    return os.cpu_count() or 1


# ------------------------------------------------------------------ stages

def dist32(a, b) -> float:
    """Canonical FP32 Euclidean distance (32 fmaf partials t mod 32, xor
    butterfly 16, 8, 4, 2, 1, sqrtf)."""
    a, b = _f32(a).ravel(), _f32(b).ravel()
    return float(_lib().or_dist32(a, b, a.size))


def dist64(a, b) -> float:
    a, b = _f32(a).ravel(), _f32(b).ravel()
    return float(_lib().or_dist64(a, b, a.size))


def knn(X, k: int, rows=None, threads: int | None = None):
    """Exact kNN (self excluded, order (w, id)). ``rows`` = (r0, r1) range
    of query rows; returns (nbr int32 [r1-r0, k], dist float32 [r1-r0, k])."""
    X = _f32(X)
    n, d = X.shape
    if not 1 <= k <= n - 1:
        raise ValueError("need 1 <= k <= n-1")
    r0, r1 = (0, n) if rows is None else rows
    nbr = np.empty((r1 - r0, k), np.int32)
    dist = np.empty((r1 - r0, k), np.float32)
    _lib().or_knn(X, n, d, k, r0, r1, nbr, dist,
                  threads if threads is not None else threads_default())
    return nbr, dist


@dataclass
class NNDescent:
    nbr: np.ndarray       # n x k ids, (w, id) ascending per row
    dist: np.ndarray      # n x k canonical distances
    iters: int            # iterations run
    updates: np.ndarray   # c of every iteration run
    pairs: np.ndarray     # pairs evaluated by the joins of every iteration


def nndescent(X, k: int, S: int, max_iters: int, delta: float, seed: int,
              init=None) -> NNDescent:
    """NN-Descent (Dong, Charikar and Li, 2011), the algorithm behind the
    paper's Phase 1 library, with set-defined steps (see ``or_nndescent``):
    lists of k, samples of S per class over both directions with Philox
    priorities, local joins, k smallest of each list and its proposals;
    stop when an iteration changes fewer than delta n k entries (or none)."""
    X = _f32(X)
    n, d = X.shape
    if not (1 <= k <= n - 1 and 1 <= S and max_iters >= 0):
        raise ValueError("need 1 <= k <= n-1, S >= 1, max_iters >= 0")
    ip = None
    if init is not None:
        init = _i32(init).reshape(n, k)
        if (init < 0).any() or (init >= n).any() or (init == np.arange(n)[:, None]).any():
            raise ValueError("init ids must be in [0, n) and not the row itself")
        if any(len(set(r)) != k for r in init.tolist()):
            raise ValueError("init rows must hold k distinct ids")
        ip = init.ctypes.data_as(ctypes.c_void_p)
    nbr = np.empty((n, k), np.int32)
    dist = np.empty((n, k), np.float32)
    upd = np.zeros(max(max_iters, 1), np.int64)
    prs = np.zeros(max(max_iters, 1), np.int64)
    it = _lib().or_nndescent(X, n, d, k, S, max_iters, float(delta), seed & (2**64 - 1), ip,
                             nbr, dist, upd, prs)
    return NNDescent(nbr, dist, int(it), upd[:it].copy(), prs[:it].copy())


def recall(nbr, exact_nbr) -> float:
    """Fraction of the exact kNN ids that a graph's rows hold (recall@k)."""
    nbr, exact_nbr = np.asarray(nbr), np.asarray(exact_nbr)
    n, k = exact_nbr.shape
    hit = 0
    for a, b in zip(nbr, exact_nbr):
        hit += len(np.intersect1d(a, b, assume_unique=True))
    return hit / (n * k)


def knn_rows(X, k: int, rows, threads: int | None = None):
    """Exact kNN for an arbitrary list of query rows (one row at a time)."""
    rows = np.asarray(rows, dtype=np.int64)
    nbr = np.empty((rows.size, k), np.int32)
    dist = np.empty((rows.size, k), np.float32)
    X = _f32(X)
    n, d = X.shape
    L = _lib()
    th = threads if threads is not None else threads_default()

    def one(q):
        r = int(rows[q])
        a = np.empty((1, k), np.int32)
        b = np.empty((1, k), np.float32)
        L.or_knn(X, n, d, k, r, r + 1, a, b, 1)  # ctypes drops the GIL here
        nbr[q] = a[0]
        dist[q] = b[0]

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, th)) as ex:
        list(ex.map(one, range(rows.size)))
    return nbr, dist


@dataclass
class Graph:
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz], sorted and unique per row

    def neighbours(self, v: int) -> np.ndarray:
        return self.col[self.row_ptr[v]:self.row_ptr[v + 1]]


def build_graph(nbr) -> Graph:
    """Undirected G from the neighbour lists (Alg. 2, first loop)."""
    nbr = _i32(nbr)
    n, k = nbr.shape
    row_ptr = np.empty(n + 1, np.int64)
    col = np.empty(max(1, 2 * n * k), np.int32)
    nnz = _lib().or_build_graph(nbr, n, k, row_ptr, col)
    return Graph(row_ptr, col[:nnz].copy())


@dataclass
class Components:
    comp: np.ndarray       # int32 [n], component index in DFS discovery order
    members: np.ndarray    # int32 [n], members grouped by component, ids ascending
    comp_off: np.ndarray   # int64 [t+1]

    @property
    def t(self) -> int:
        return self.comp_off.size - 1

    def sizes(self) -> np.ndarray:
        return np.diff(self.comp_off)


def components(G: Graph) -> Components:
    """Depth-first search components of G (Alg. 2)."""
    n = G.row_ptr.size - 1
    comp = np.empty(n, np.int32)
    members = np.empty(n, np.int32)
    off = np.empty(n + 1, np.int64)
    t = _lib().or_components(n, G.row_ptr, np.ascontiguousarray(G.col), comp,
                             members, off)
    return Components(comp, members, off[:t + 1].copy())


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    _lib().or_philox4x32_10(c, k, out)
    return out


@dataclass
class Edges:
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    ci: np.ndarray
    cj: np.ndarray

    def copy(self) -> "Edges":
        return Edges(self.u.copy(), self.v.copy(), self.w.copy(),
                     self.ci.copy(), self.cj.copy())

    def __len__(self):
        return int(self.u.size)


def random_edges(X, C: Components, lam: int, seed: int) -> Edges:
    """lambda shortest of lambda^2 random samples per component pair (Alg. 3)."""
    X = _f32(X)
    n, d = X.shape
    t = C.t
    m = lam * t * (t - 1) // 2
    out = [np.empty(max(1, m), dt) for dt in
           (np.int32, np.int32, np.float32, np.int32, np.int32)]
    got = _lib().or_random_edges(X, d, C.members, C.comp_off, t, lam,
                                 np.uint64(seed), *out)
    assert got == m
    return Edges(*(a[:m].copy() for a in out))


def nearest_edges(X, C: Components, lam: int) -> Edges:
    """The lambda nearest pairs (u in C_i, v in C_j) of every component pair
    under the order (w, min id, max id): the nearest-pair variant of Alg. 3."""
    X = _f32(X)
    n, d = X.shape
    t = C.t
    m = lam * t * (t - 1) // 2
    out = [np.empty(max(1, m), dt) for dt in
           (np.int32, np.int32, np.float32, np.int32, np.int32)]
    got = _lib().or_nearest_edges(X, d, C.members, C.comp_off, t, lam, *out)
    assert got == m
    return Edges(*(a[:m].copy() for a in out))


def refine_sweep(X, G: Graph, C: Components, E: Edges, changed=None) -> int:
    """One sweep of Alg. 4 over E, in place; returns |Delta|."""
    X = _f32(X)
    d = X.shape[1]
    m = len(E)
    ch = np.zeros(max(1, m), np.uint8) if changed is None else changed
    return int(_lib().or_refine_sweep(X, d, G.row_ptr, np.ascontiguousarray(G.col),
                                      C.comp, m, E.u, E.v, E.w, E.ci, E.cj, ch))


def refine(X, G: Graph, C: Components, E: Edges, max_iters: int = 10000):
    """Repeat Alg. 4 until |Delta| = 0 (Alg. 1). Returns the list of |Delta|
    per sweep (its last entry is 0 unless the cap was hit) and, per edge, the
    number of sweeps in which it changed."""
    deltas = []
    changes = np.zeros(len(E), np.int64)
    ch = np.zeros(max(1, len(E)), np.uint8)
    for _ in range(max_iters):
        dl = refine_sweep(X, G, C, E, ch)
        changes += ch[:len(E)]
        deltas.append(dl)
        if dl == 0:
            break
    return deltas, changes


@dataclass
class Tree:
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    W: float

    def key_sorted(self):
        """Edges as (w, min, max) sorted by that key (a canonical form)."""
        a = np.minimum(self.u, self.v)
        b = np.maximum(self.u, self.v)
        o = np.lexsort((b, a, self.w))
        return self.w[o], a[o], b[o]


def kruskal(n: int, nbr, dist, E: Edges | None) -> Tree:
    nbr = _i32(nbr)
    dist = _f32(dist)
    k = nbr.shape[1] if nbr.ndim == 2 else 0
    if E is None:
        E = Edges(*(np.zeros(0, dt) for dt in
                    (np.int32, np.int32, np.float32, np.int32, np.int32)))
    tu = np.empty(max(1, n - 1), np.int32)
    tv = np.empty(max(1, n - 1), np.int32)
    tw = np.empty(max(1, n - 1), np.float32)
    W = ctypes.c_double(0.0)
    eu = E.u if len(E) else np.zeros(1, np.int32)
    ev = E.v if len(E) else np.zeros(1, np.int32)
    ew = E.w if len(E) else np.zeros(1, np.float32)
    got = _lib().or_kruskal(n, nbr if nbr.size else np.zeros(1, np.int32),
                            dist if dist.size else np.zeros(1, np.float32), k,
                            len(E), _i32(eu), _i32(ev), _f32(ew), tu, tv, tw,
                            ctypes.byref(W))
    return Tree(tu[:got].copy(), tv[:got].copy(), tw[:got].copy(), W.value)


def prim_exact(X, threads: int | None = None) -> Tree:
    """Exact MST of the complete graph by O(n^2) Prim (plays the EMST role)."""
    X = _f32(X)
    n, d = X.shape
    tu = np.empty(max(1, n - 1), np.int32)
    tv = np.empty(max(1, n - 1), np.int32)
    tw = np.empty(max(1, n - 1), np.float32)
    W = ctypes.c_double(0.0)
    _lib().or_prim(X, n, d, tu, tv, tw, ctypes.byref(W),
                   threads if threads is not None else threads_default())
    m = max(0, n - 1)
    return Tree(tu[:m].copy(), tv[:m].copy(), tw[:m].copy(), W.value)


def tree_weight64(X, tu, tv) -> float:
    X = _f32(X)
    return float(_lib().or_tree_weight64(X, X.shape[1], _i32(tu), _i32(tv),
                                         int(np.asarray(tu).size)))


def mst_grad(X, tu, tv) -> np.ndarray:
    X = _f32(X)
    n, d = X.shape
    g = np.empty((n, d), np.float64)
    _lib().or_mst_grad(X, n, d, _i32(tu), _i32(tv), int(np.asarray(tu).size), g)
    return g


def relative_error(W_approx: float, W_exact: float) -> float:
    """Eq. 1."""
    return (W_approx - W_exact) / W_exact


@dataclass
class FamstResult:
    nbr: np.ndarray
    dist: np.ndarray
    G: Graph
    C: Components
    E0: Edges            # edges as Alg. 3 produced them
    E: Edges             # edges after refinement
    deltas: list = field(default_factory=list)
    changes: np.ndarray | None = None
    tree: Tree | None = None


def famst(X, k: int, lam: int, seed: int, knn_graph=None,
          max_iters: int = 10000, threads: int | None = None,
          connect: str = "random", nnd: dict | None = None) -> FamstResult:
    """Algorithm 1. ``knn_graph`` = (nbr, dist) replaces the exact kNN stage
    (used to run the later stages on another implementation's graph);
    ``connect`` = "random" (Alg. 3) or "nearest" (the lambda nearest pairs
    of every component pair); ``nnd`` = dict(S=, max_iters=, delta=) takes
    Phase 1 by NN-Descent with the build's seed."""
    X = _f32(X)
    n = X.shape[0]
    if knn_graph is None and nnd is not None:
        r = nndescent(X, k, nnd["S"], nnd["max_iters"], nnd["delta"], seed)
        nbr, dist = r.nbr, r.dist
    elif knn_graph is None:
        nbr, dist = knn(X, k, threads=threads)
    else:
        nbr, dist = _i32(knn_graph[0]), _f32(knn_graph[1])
    G = build_graph(nbr)
    C = components(G)
    E0 = nearest_edges(X, C, lam) if connect == "nearest" else random_edges(X, C, lam, seed)
    E = E0.copy()
    deltas, changes = refine(X, G, C, E, max_iters=max_iters)
    tree = kruskal(n, nbr, dist, E)
    return FamstResult(nbr, dist, G, C, E0, E, deltas, changes, tree)
