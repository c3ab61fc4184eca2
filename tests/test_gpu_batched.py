"""famst_build_batched: many clouds of uneven n and d in one call. Each
cloud's tree must be bit-identical to famst_build of that cloud alone with
seed + b (the batch shares no data between clouds), the second identical
call replays the captured CUDA graph with the same output, and the oracle
agrees on sampled clouds."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - deselected on CPU runs
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_14261_gb300 as P
    return P.Context(0)


def _concat(clouds):
    offsets = np.zeros(len(clouds) + 1, np.int64)
    for b, c in enumerate(clouds):
        offsets[b + 1] = offsets[b] + c.shape[0]
    dims = np.array([c.shape[1] for c in clouds], np.int32)
    flat = np.concatenate([c.ravel() for c in clouds]).astype(np.float32)
    return torch.from_numpy(flat).cuda(), offsets, dims


def _small_batch():
    return workloads.batch_clouds(count=12, base_seed=2000, n_range=(300, 2500))


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_batched_equals_single_builds(ctx, prec):
    clouds = _small_batch()
    Xc, off, dims = _concat(clouds)
    k, lam, seed = 16, 5, 77
    trees, W, t, info = ctx.build_batched(Xc, off, dims, k, lam, seed, prec)
    import paper_2507_14261_gb300 as P
    assert info.graph_replayed == 0
    assert info.graph_kernels > 0, P.lib().famst_last_error(ctx._h)
    for b, c in enumerate(clouds):
        single, sinfo = ctx.build(torch.from_numpy(c).cuda(), k, lam, seed + b, prec)
        assert torch.equal(trees[b].u, single.u) and torch.equal(trees[b].v, single.v)
        assert torch.equal(trees[b].w, single.w)
        assert W[b] == pytest.approx(single.W, rel=1e-12)
        assert t[b] == sinfo.t
    # the same call again replays the captured graph, bit for bit
    trees2, W2, t2, info2 = ctx.build_batched(Xc, off, dims, k, lam, seed, prec)
    assert info2.graph_replayed == 1 and info2.graph_kernels > 0
    for b in range(len(clouds)):
        assert torch.equal(trees2[b].u, trees[b].u) and torch.equal(trees2[b].w, trees[b].w)
    assert np.array_equal(W2, W) and np.array_equal(t2, t)


def test_batched_matches_oracle(orc, ctx):
    clouds = _small_batch()[:4]
    Xc, off, dims = _concat(clouds)
    trees, W, t, info = ctx.build_batched(Xc, off, dims, 10, 3, 5, "bf16x3")
    for b, c in enumerate(clouds):
        ref = orc.famst(c, 10, 3, 5 + b)
        got = sorted(zip(trees[b].w.cpu().tolist(),
                         np.minimum(trees[b].u.cpu(), trees[b].v.cpu()).tolist(),
                         np.maximum(trees[b].u.cpu(), trees[b].v.cpu()).tolist()))
        want = sorted(zip(ref.tree.w.tolist(), np.minimum(ref.tree.u, ref.tree.v).tolist(),
                          np.maximum(ref.tree.u, ref.tree.v).tolist()))
        assert got == want
        assert W[b] == pytest.approx(ref.tree.W, rel=1e-12)
        assert t[b] == ref.C.t


def test_batched_capacity_retry(ctx):
    # a cloud of 70 tight, well separated clusters has more components than
    # the first capacity guess; the call must size up and still be exact
    many = workloads.blobs(70 * 24, 8, 70, (0.05, 0.05), 31)
    clouds = [many, workloads.blobs(900, 3, 5, (1, 1), 32)]
    Xc, off, dims = _concat(clouds)
    trees, W, t, info = ctx.build_batched(Xc, off, dims, 6, 2, 9, "bf16x3")
    assert t[0] > 48
    single, sinfo = ctx.build(torch.from_numpy(many).cuda(), 6, 2, 9, "bf16x3")
    assert torch.equal(trees[0].u, single.u) and torch.equal(trees[0].w, single.w)
