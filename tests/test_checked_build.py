"""The bounds-checked debug build (libfamst_checked.so: the C ABI compiled
with FAMST_CHECK_BOUNDS). Between the stages of a build it validates every
index array on the device -- kNN ids, component labels, member lists,
inter-component edges after Alg. 3 and Alg. 4, tree edges -- and fails the
call, without a fault, if one is out of range. Here: it builds and exports
the same entry points (CPU), and on the GPU a checked build raises no
alarm and returns the release library's tree bit for bit."""
import ctypes

import numpy as np
import pytest

import workloads
from test_abi import declared_functions


def test_checked_library_builds_and_exports_everything():
    from paper_2507_14261_gb300 import _build_lib
    L = ctypes.CDLL(_build_lib.build_checked())
    missing = [nm for nm in declared_functions() if not hasattr(L, nm)]
    assert not missing, missing


@pytest.mark.gpu
def test_checked_build_matches_release_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover - deselected on CPU runs
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_14261_gb300 as P
    from paper_2507_14261_gb300 import _build_lib
    L = ctypes.CDLL(_build_lib.build_checked())
    P_ = ctypes.c_void_p
    L.famst_create.argtypes = [ctypes.POINTER(P_), ctypes.c_int]
    L.famst_destroy.argtypes = [P_]
    L.famst_last_error.argtypes = [P_]
    L.famst_last_error.restype = ctypes.c_char_p
    L.famst_build.argtypes = [P_, P_, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                              P_, P_, P_, ctypes.POINTER(ctypes.c_double), P_]
    for X in (workloads.blobs(3000, 64, 20, (0.5, 1.5), 81),        # BF16 staged refinement
              workloads.blobs(2000, 3, 12, (0.2, 0.6), 82)):        # FP32 filters
        n, d = X.shape
        Xd = torch.from_numpy(X).cuda()
        ref, _ = P.Context(0).build(Xd, 8, 5, 3, "bf16x3")
        h = P_()
        assert L.famst_create(ctypes.byref(h), 0) == 0
        try:
            tu = torch.empty(n - 1, dtype=torch.int32, device="cuda")
            tv = torch.empty_like(tu)
            tw = torch.empty(n - 1, dtype=torch.float32, device="cuda")
            W = ctypes.c_double(0.0)
            torch.cuda.synchronize()
            st = L.famst_build(h, P_(Xd.data_ptr()), n, d, 8, 5, 3, 2, 10000,
                               P_(tu.data_ptr()), P_(tv.data_ptr()), P_(tw.data_ptr()),
                               ctypes.byref(W), None)
            assert st == 0, L.famst_last_error(h)
        finally:
            L.famst_destroy(h)
        assert torch.equal(tu, ref.u) and torch.equal(tv, ref.v) and torch.equal(tw, ref.w)
        assert W.value == ref.W
