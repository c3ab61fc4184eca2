"""Python binding of the FAMST C ABI (include/famst.h).

Argument marshalling only: every step of the method runs in the CUDA
library ``libfamst.so``. PyTorch supplies device memory (tensors) and the
current CUDA stream. If the library is missing the calls raise; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build_lib

FAMST_OK = 0
ERRORS = {
    -1: "FAMST_ERR_INVALID_ARG", -2: "FAMST_ERR_CAPACITY", -3: "FAMST_ERR_NO_CONVERGENCE",
    -4: "FAMST_ERR_TIMEOUT", -5: "FAMST_ERR_CUDA", -6: "FAMST_ERR_OOM",
    -7: "FAMST_ERR_UNSUPPORTED", -8: "FAMST_ERR_NONFINITE", -9: "FAMST_ERR_DISCONNECTED",
}
PREC = {"fp32": 0, "bf16": 1, "bf16x3": 2, "fp8": 3}


class FamstError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{ERRORS.get(status, status)}: {detail}")
        self.status = status
        self.name = ERRORS.get(status, str(status))


class BuildInfo(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_int64), ("m", ctypes.c_int64), ("refine_sweeps", ctypes.c_int32),
        ("boruvka_rounds", ctypes.c_int32), ("first_delta", ctypes.c_int64),
        ("uncertified_rows", ctypes.c_int64), ("W", ctypes.c_double), ("W64", ctypes.c_double),
        ("ms_knn", ctypes.c_double), ("ms_components", ctypes.c_double),
        ("ms_connect", ctypes.c_double), ("ms_refine", ctypes.c_double),
        ("ms_mst", ctypes.c_double), ("ms_total", ctypes.c_double),
        ("knn_tile_fraction", ctypes.c_double), ("refine_distance_evals", ctypes.c_int64),
        ("refine_canonical_evals", ctypes.c_int64), ("refine_filter", ctypes.c_int32),
        ("knn_iters", ctypes.c_int32), ("ms_knn_tiles", ctypes.c_double),
        ("ms_rerank", ctypes.c_double), ("ms_connect_kernel", ctypes.c_double),
        ("ms_refine_kernel", ctypes.c_double), ("refine_rows_staged", ctypes.c_int64),
        ("refine_fixed_rows", ctypes.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("refine_sweeps", ctypes.c_int32),
        ("boruvka_rounds", ctypes.c_int32), ("uncertified_rows", ctypes.c_int64),
        ("tensor_clouds", ctypes.c_int32), ("graph_replayed", ctypes.c_int32),
        ("graph_kernels", ctypes.c_int64), ("tile_epilogue_warps", ctypes.c_int32),
        ("tile_stages", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_F32 = ctypes.c_float
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PD = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "famst_create": (_I32, [ctypes.POINTER(_P), ctypes.c_int]),
    "famst_destroy": (_I32, [_P]),
    "famst_set_stream": (_I32, [_P, _P]),
    "famst_set_knn_pruning": (_I32, [_P, _I32]),
    "famst_set_loop_limit": (_I32, [_P, _I32]),
    "famst_set_connect_mode": (_I32, [_P, _I32]),
    "famst_connect_nearest": (_I32, [_P, _P, _I64, _I32, _P, _I64, _I32, _P, _P, _P, _P, _P,
                                     _I64, _PI64]),
    "famst_workspace_query": (_I32, [_P, _I64, _I32, _I32, _I32, _I64, _I32, _I32,
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "famst_error_string": (ctypes.c_char_p, [_I32]),
    "famst_last_error": (ctypes.c_char_p, [_P]),
    "famst_launch_count": (ctypes.c_uint64, [_P]),
    "famst_workspace_bytes": (ctypes.c_size_t, [_P]),
    "famst_knn_graph": (_I32, [_P, _P, _I64, _I32, _I32, _I32, _P, _P]),
    "famst_knn_nndescent": (_I32, [_P, _P, _I64, _I32, _I32, _I32, _I32, ctypes.c_double, _U64,
                                   _P, _P, _P, _PI32, _P, _P]),
    "famst_set_knn_method": (_I32, [_P, _I32, _I32, _I32, ctypes.c_double]),
    "famst_components": (_I32, [_P, _P, _I64, _I32, _P, _PI64]),
    "famst_connect": (_I32, [_P, _P, _I64, _I32, _P, _I64, _I32, _U64, _P, _P, _P, _P, _P,
                             _I64, _PI64]),
    "famst_refine": (_I32, [_P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _P, _P, _P, _I64, _I32,
                            _PI32, _PI64]),
    "famst_mst": (_I32, [_P, _I64, _P, _P, _I32, _P, _P, _P, _I64, _P, _P, _P, _PD]),
    "famst_tree_weight": (_I32, [_P, _P, _I64, _I32, _P, _P, _P, _I64, _PD, _PD]),
    "famst_build": (_I32, [_P, _P, _I64, _I32, _I32, _I32, _U64, _I32, _I32, _P, _P, _P, _PD,
                           ctypes.POINTER(BuildInfo)]),
    "famst_build_host": (_I32, [_P, _P, _I64, _I32, _I32, _I32, _U64, _I32, _I32, _P, _P, _P,
                                _PD, ctypes.POINTER(BuildInfo)]),
    "famst_mst_backward": (_I32, [_P, _P, _I64, _I32, _P, _P, _I64, _F32, _P]),
    "famst_emst_exact": (_I32, [_P, _P, _I64, _I32, _I32, _P, _P, _P, _PD, _PI32]),
    "famst_build_batched": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _U64, _I32, _I32, _P, _P,
                                   _P, _P, _P, ctypes.POINTER(BatchInfo)]),
}


def library_path() -> str:
    return _build_lib.lib_path()


def lib():
    """Load libfamst.so (built by ``__graft_entry__.build()``)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"the FAMST CUDA library is not built ({path}); "
                               "run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, name: str, cuda: bool = True):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if cuda and not t.is_cuda:
        raise TypeError(f"{name} must be on a CUDA device")


class Context:
    """A library context bound to one CUDA device; work goes to the torch
    stream current at each call."""

    def __init__(self, device: int | None = None):
        L = lib()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = ctypes.c_void_p()
        st = L.famst_create(ctypes.byref(h), device)
        if st != FAMST_OK:
            raise FamstError(st, "famst_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().famst_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------- helpers
    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        lib().famst_set_stream(self._h, ctypes.c_void_p(s))

    def _check(self, st: int, what: str):
        if st != FAMST_OK:
            detail = lib().famst_last_error(self._h)
            raise FamstError(st, f"{what}: {detail.decode() if detail else ''}")

    @property
    def launches(self) -> int:
        return int(lib().famst_launch_count(self._h))

    @property
    def workspace_bytes(self) -> int:
        return int(lib().famst_workspace_bytes(self._h))

    def set_loop_limit(self, limit: int):
        """Iteration limit of the union-find and Boruvka loops (0 = defaults);
        a loop that reaches it makes the call raise FAMST_ERR_TIMEOUT."""
        self._check(lib().famst_set_loop_limit(self._h, int(limit)), "famst_set_loop_limit")

    def workspace_query(self, n: int, d: int, k: int, lam: int, t_max: int,
                        prec: str = "fp32", max_iters: int = 10000) -> int:
        """Device workspace bytes a build of this shape needs (at most t_max
        components in its kNN graph)."""
        b = ctypes.c_size_t(0)
        self._check(lib().famst_workspace_query(self._h, n, d, k, lam, t_max, PREC[prec],
                                                max_iters, ctypes.byref(b)),
                    "famst_workspace_query")
        return int(b.value)

    def set_knn_pruning(self, enable: bool):
        """Phase 1 tile pruning on (default) or off; the kNN graph is exact
        either way."""
        self._check(lib().famst_set_knn_pruning(self._h, 1 if enable else 0),
                    "famst_set_knn_pruning")

    # ----------------------------------------------------------- phases
    def knn_graph(self, X: torch.Tensor, k: int, prec: str = "fp32"):
        _need(X, torch.float32, "X")
        n, d = X.shape
        nbr = torch.empty((n, k), dtype=torch.int32, device=X.device)
        dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
        self._stream()
        st = lib().famst_knn_graph(self._h, _ptr(X), n, d, k, PREC[prec], _ptr(nbr), _ptr(dist))
        self._check(st, "famst_knn_graph")
        return nbr, dist

    def knn_nndescent(self, X: torch.Tensor, k: int, S: int | None = None, max_iters: int = 10,
                      delta: float = 0.001, seed: int = 0, init=None):
        """famst_knn_nndescent: approximate kNN graph by NN-Descent. Returns
        (nbr, dist, iterations, updates per iteration, join pairs per
        iteration)."""
        import numpy as np
        _need(X, torch.float32, "X")
        n, d = X.shape
        S = min(k, 32) if S is None else S
        if init is not None:
            _need(init, torch.int32, "init")
        nbr = torch.empty((n, k), dtype=torch.int32, device=X.device)
        dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
        it = ctypes.c_int32(0)
        upd = np.zeros(max(max_iters, 1), np.int64)
        prs = np.zeros(max(max_iters, 1), np.int64)
        self._stream()
        st = lib().famst_knn_nndescent(self._h, _ptr(X), n, d, k, S, max_iters, float(delta),
                                       seed & (2**64 - 1), _ptr(init) if init is not None else None,
                                       _ptr(nbr), _ptr(dist), ctypes.byref(it),
                                       upd.ctypes.data_as(ctypes.c_void_p),
                                       prs.ctypes.data_as(ctypes.c_void_p))
        self._check(st, "famst_knn_nndescent")
        return nbr, dist, int(it.value), upd[:it.value].copy(), prs[:it.value].copy()

    def set_knn_method(self, method: str, S: int = 0, max_iters: int = 10, delta: float = 0.001):
        """Phase 1 of builds: "exact" (tiles) or "nndescent"."""
        code = {"exact": 0, "nndescent": 1}[method]
        self._check(lib().famst_set_knn_method(self._h, code, S, max_iters, float(delta)),
                    "famst_set_knn_method")

    def components(self, nbr: torch.Tensor):
        _need(nbr, torch.int32, "nbr")
        n, k = nbr.shape
        comp = torch.empty(n, dtype=torch.int32, device=nbr.device)
        t = ctypes.c_int64(0)
        self._stream()
        st = lib().famst_components(self._h, _ptr(nbr), n, k, _ptr(comp), ctypes.byref(t))
        self._check(st, "famst_components")
        return comp, int(t.value)

    def connect(self, X, comp, t: int, lam: int, seed: int, capacity: int | None = None):
        _need(X, torch.float32, "X")
        _need(comp, torch.int32, "comp")
        n, d = X.shape
        m = lam * t * (t - 1) // 2
        cap = m if capacity is None else capacity
        dev = X.device
        E = Edges(*(torch.empty(max(cap, 1), dtype=dt, device=dev) for dt in
                    (torch.int32, torch.int32, torch.float32, torch.int32, torch.int32)))
        mo = ctypes.c_int64(0)
        self._stream()
        st = lib().famst_connect(self._h, _ptr(X), n, d, _ptr(comp), t, lam, seed & (2**64 - 1),
                                 _ptr(E.u), _ptr(E.v), _ptr(E.w), _ptr(E.ci), _ptr(E.cj), cap,
                                 ctypes.byref(mo))
        if st == -2:
            raise FamstError(st, f"capacity {cap} < required {mo.value}")
        self._check(st, "famst_connect")
        return E.slice(int(mo.value))

    def connect_nearest(self, X, comp, t: int, lam: int, capacity: int | None = None):
        """famst_connect_nearest: the lambda nearest pairs of every component
        pair (order (w, min id, max id)), in famst_connect's layout."""
        _need(X, torch.float32, "X")
        _need(comp, torch.int32, "comp")
        n, d = X.shape
        m = lam * t * (t - 1) // 2
        cap = m if capacity is None else capacity
        dev = X.device
        E = Edges(*(torch.empty(max(cap, 1), dtype=dt, device=dev) for dt in
                    (torch.int32, torch.int32, torch.float32, torch.int32, torch.int32)))
        mo = ctypes.c_int64(0)
        self._stream()
        st = lib().famst_connect_nearest(self._h, _ptr(X), n, d, _ptr(comp), t, lam, _ptr(E.u),
                                         _ptr(E.v), _ptr(E.w), _ptr(E.ci), _ptr(E.cj), cap,
                                         ctypes.byref(mo))
        if st == -2:
            raise FamstError(st, f"capacity {cap} < required {mo.value}")
        self._check(st, "famst_connect_nearest")
        return E.slice(int(mo.value))

    def set_connect_mode(self, mode: str):
        """Connect step of builds: "random" (Algorithm 3) or "nearest"."""
        code = {"random": 0, "nearest": 1}[mode]
        self._check(lib().famst_set_connect_mode(self._h, code), "famst_set_connect_mode")

    def refine(self, X, nbr, comp, E: "Edges", max_iters: int = 10000):
        _need(X, torch.float32, "X")
        _need(nbr, torch.int32, "nbr")
        n, d = X.shape
        k = nbr.shape[1]
        sweeps = ctypes.c_int32(0)
        hist = (ctypes.c_int64 * max_iters)()
        self._stream()
        st = lib().famst_refine(self._h, _ptr(X), n, d, _ptr(nbr), k, _ptr(comp), _ptr(E.u),
                                _ptr(E.v), _ptr(E.w), _ptr(E.ci), _ptr(E.cj), len(E), max_iters,
                                ctypes.byref(sweeps), hist)
        self._check(st, "famst_refine")
        s = int(sweeps.value)
        return s, [int(hist[i]) for i in range(s)]

    def mst(self, n: int, nbr, dist, E: "Edges | None"):
        _need(nbr, torch.int32, "nbr")
        _need(dist, torch.float32, "dist")
        k = nbr.shape[1]
        dev = nbr.device
        tu = torch.empty(max(n - 1, 1), dtype=torch.int32, device=dev)
        tv = torch.empty_like(tu)
        tw = torch.empty(max(n - 1, 1), dtype=torch.float32, device=dev)
        W = ctypes.c_double(0)
        m = 0 if E is None else len(E)
        self._stream()
        st = lib().famst_mst(self._h, n, _ptr(nbr), _ptr(dist), k,
                             _ptr(E.u) if m else None, _ptr(E.v) if m else None,
                             _ptr(E.w) if m else None, m, _ptr(tu), _ptr(tv), _ptr(tw),
                             ctypes.byref(W))
        self._check(st, "famst_mst")
        return tu[: n - 1], tv[: n - 1], tw[: n - 1], W.value

    def emst_exact(self, X, prec: str = "bf16x3"):
        """Exact EMST of the complete graph (the tree T* of Eq. 1) by Boruvka
        rounds over masked exact 1-NN passes. Returns (Tree, rounds)."""
        _need(X, torch.float32, "X")
        n, d = X.shape
        dev = X.device
        tu = torch.empty(max(n - 1, 1), dtype=torch.int32, device=dev)
        tv = torch.empty_like(tu)
        tw = torch.empty(max(n - 1, 1), dtype=torch.float32, device=dev)
        W = ctypes.c_double(0)
        rounds = ctypes.c_int32(0)
        self._stream()
        st = lib().famst_emst_exact(self._h, _ptr(X), n, d, PREC[prec], _ptr(tu), _ptr(tv),
                                    _ptr(tw), ctypes.byref(W), ctypes.byref(rounds))
        self._check(st, "famst_emst_exact")
        return Tree(tu[: n - 1], tv[: n - 1], tw[: n - 1], W.value), rounds.value

    def tree_weight(self, X, tu, tv, tw):
        n, d = X.shape
        W = ctypes.c_double(0)
        W64 = ctypes.c_double(0)
        self._stream()
        st = lib().famst_tree_weight(self._h, _ptr(X), n, d, _ptr(tu), _ptr(tv), _ptr(tw),
                                     tu.numel(), ctypes.byref(W), ctypes.byref(W64))
        self._check(st, "famst_tree_weight")
        return W.value, W64.value

    def build(self, X, k: int, lam: int, seed: int = 0, prec: str = "fp32",
              max_iters: int = 10000):
        _need(X, torch.float32, "X")
        n, d = X.shape
        dev = X.device
        tu = torch.empty(max(n - 1, 1), dtype=torch.int32, device=dev)
        tv = torch.empty_like(tu)
        tw = torch.empty(max(n - 1, 1), dtype=torch.float32, device=dev)
        W = ctypes.c_double(0)
        info = BuildInfo()
        self._stream()
        st = lib().famst_build(self._h, _ptr(X), n, d, k, lam, seed & (2**64 - 1), PREC[prec],
                               max_iters, _ptr(tu), _ptr(tv), _ptr(tw), ctypes.byref(W),
                               ctypes.byref(info))
        self._check(st, "famst_build")
        return Tree(tu[: n - 1], tv[: n - 1], tw[: n - 1], W.value), info

    def build_host(self, X_host, k: int, lam: int, seed: int = 0, prec: str = "fp32",
                   max_iters: int = 10000, out=None):
        """famst_build_host: X and the tree in host memory (pin them for
        fast copies). ``out`` = preallocated (tu, tv, tw) host tensors."""
        _need(X_host, torch.float32, "X_host", cuda=False)
        n, d = X_host.shape
        if out is None:
            out = (torch.empty(max(n - 1, 1), dtype=torch.int32),
                   torch.empty(max(n - 1, 1), dtype=torch.int32),
                   torch.empty(max(n - 1, 1), dtype=torch.float32))
        tu, tv, tw = out
        W = ctypes.c_double(0)
        info = BuildInfo()
        self._stream()
        st = lib().famst_build_host(self._h, _ptr(X_host), n, d, k, lam, seed & (2**64 - 1),
                                    PREC[prec], max_iters, _ptr(tu), _ptr(tv), _ptr(tw),
                                    ctypes.byref(W), ctypes.byref(info))
        self._check(st, "famst_build_host")
        return Tree(tu[: n - 1], tv[: n - 1], tw[: n - 1], W.value), info

    def build_batched(self, X_concat, offsets, dims, k: int, lam: int, seed: int = 0,
                      prec: str = "bf16x3", max_iters: int = 10000, out=None):
        """famst_build_batched. X_concat: 1-D float32 device tensor holding
        the clouds back to back (cloud b: n_b x dims[b], row-major);
        offsets: B+1 point offsets; dims: B. Returns per-cloud trees (views
        of one edge array with cloud-local ids), W per cloud, t per cloud
        and the BatchInfo."""
        import numpy as np
        _need(X_concat, torch.float32, "X_concat")
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        dm = np.ascontiguousarray(dims, dtype=np.int32)
        B = dm.size
        N = int(off[-1])
        dev = X_concat.device
        if out is None:
            out = (torch.empty(max(N - B, 1), dtype=torch.int32, device=dev),
                   torch.empty(max(N - B, 1), dtype=torch.int32, device=dev),
                   torch.empty(max(N - B, 1), dtype=torch.float32, device=dev))
        tu, tv, tw = out
        W = np.zeros(B, np.float64)
        t = np.zeros(B, np.int64)
        info = BatchInfo()
        self._stream()
        st = lib().famst_build_batched(
            self._h, _ptr(X_concat), off.ctypes.data_as(ctypes.c_void_p),
            dm.ctypes.data_as(ctypes.c_void_p), B, k, lam, seed & (2**64 - 1), PREC[prec],
            max_iters, _ptr(tu), _ptr(tv), _ptr(tw), W.ctypes.data_as(ctypes.c_void_p),
            t.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
        self._check(st, "famst_build_batched")
        trees = []
        for b in range(B):
            a, e = int(off[b]) - b, int(off[b + 1]) - b - 1
            trees.append(Tree(tu[a:e], tv[a:e], tw[a:e], float(W[b])))
        return trees, W, t, info

    def mst_backward(self, X, tu, tv, gW: float = 1.0, out=None):
        _need(X, torch.float32, "X")
        n, d = X.shape
        gX = torch.empty_like(X) if out is None else out
        self._stream()
        st = lib().famst_mst_backward(self._h, _ptr(X), n, d, _ptr(tu), _ptr(tv), tu.numel(),
                                      float(gW), _ptr(gX))
        self._check(st, "famst_mst_backward")
        return gX


@dataclass
class Edges:
    u: torch.Tensor
    v: torch.Tensor
    w: torch.Tensor
    ci: torch.Tensor
    cj: torch.Tensor

    def __len__(self):
        return int(self.u.numel())

    def slice(self, m: int) -> "Edges":
        return Edges(self.u[:m], self.v[:m], self.w[:m], self.ci[:m], self.cj[:m])

    def clone(self) -> "Edges":
        return Edges(*(t.clone() for t in (self.u, self.v, self.w, self.ci, self.cj)))


@dataclass
class Tree:
    u: torch.Tensor
    v: torch.Tensor
    w: torch.Tensor
    W: float


_DEFAULT: dict[int, Context] = {}


def default_context(device: int | None = None) -> Context:
    if device is None:
        device = torch.cuda.current_device()
    if device not in _DEFAULT:
        _DEFAULT[device] = Context(device)
    return _DEFAULT[device]


class MSTWeight(torch.autograd.Function):
    """W(X) = total weight of the FAMST tree of X; backward holds the tree
    fixed and calls the CUDA backward kernel (0-dimensional topological
    loss: dW/dx_i = sum over tree edges at i of (x_i - x_j)/||x_i - x_j||)."""

    @staticmethod
    def forward(ctx, X, k: int, lam: int, seed: int = 0, prec: str = "fp32"):
        c = default_context(X.device.index)
        tree, _ = c.build(X.detach().contiguous(), k, lam, seed, prec)
        ctx.save_for_backward(X, tree.u, tree.v)
        return X.new_tensor(tree.W, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gW):
        X, tu, tv = ctx.saved_tensors
        c = default_context(X.device.index)
        g = c.mst_backward(X.detach().contiguous(), tu, tv, float(gW))
        return g, None, None, None, None


def mst_weight(X, k: int, lam: int, seed: int = 0, prec: str = "fp32"):
    return MSTWeight.apply(X, k, lam, seed, prec)
