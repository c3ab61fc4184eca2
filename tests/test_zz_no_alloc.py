"""famst_components_noalloc, the allocation-free variant of famst_components
for callers that must not allocate device memory (hosts that own all of it
through their own pool, loops that cannot afford cudaMalloc's implicit
synchronisation). Called through the C ABI and compared with
famst_components on two calls in a row; the labels are integers, so they
must be identical. Kept in a file collected last."""
import ctypes

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - deselected on CPU runs
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_14261_gb300 as P
    L = P.lib()
    f = L.famst_components_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return P, L


def _noalloc(L, nbr):
    n, k = nbr.shape
    comp = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    t = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st = L.famst_components_noalloc(ctypes.c_void_p(nbr.data_ptr()), n, k,
                                    ctypes.c_void_p(comp.data_ptr()),
                                    ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(s))
    assert st == 0
    torch.cuda.synchronize()
    return comp, int(t.item())


def test_noalloc_matches_components_twice(lib):
    P, L = lib
    ctx = P.Context(0)
    cases = [workloads.blobs(3000, 16, 12, (0.3, 0.6), 21),   # many components
             workloads.blobs(1700, 8, 3, (1.0, 1.0), 22)]     # fewer, smaller n
    for X in cases:
        nbr, _ = ctx.knn_graph(torch.from_numpy(X).cuda(), 4)
        want_comp, want_t = ctx.components(nbr)
        comp, t = _noalloc(L, nbr)
        assert t == want_t
        assert torch.equal(comp, want_comp)
    assert want_t >= 1


def test_noalloc_rejects_bad_sizes_and_ids(lib):
    P, L = lib
    big = 1 << 20
    nbr = torch.zeros((1, 1), dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.famst_components_noalloc(ctypes.c_void_p(nbr.data_ptr()), big + 1, 1,
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert st == -7  # FAMST_ERR_UNSUPPORTED
    bad = torch.tensor([[1], [5]], dtype=torch.int32, device="cuda")  # id 5 >= n
    comp, t = _noalloc(L, bad)
    assert t == -1
    good = torch.tensor([[1], [0], [1]], dtype=torch.int32, device="cuda")
    comp, t = _noalloc(L, good)
    assert t == 1 and comp.tolist() == [0, 0, 0]
