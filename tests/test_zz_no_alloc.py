"""The allocation-free table gather, through the C ABI.

cc_table_gather_noalloc exists for callers that cannot allocate device memory
(a framework that owns all of it through its own pool, a latency-bound loop
where cudaMalloc/cudaFree are not acceptable, a fixed memory budget).  It keeps
its scratch in a fixed file-scope device array instead of the context arena.
These checks run it twice in a row on different inputs (so the second call
would see anything the first left behind in the shared array) and compare each
result bit for bit with cc_table_gather on the same inputs and with the
oracle's neighbour sum (Eq. 1's sum over u in N(v)); integer sums have no
tolerance.  They also check that a call leaves the device's free memory and
torch's allocations unchanged, and that both entry points refuse a decreasing
row_ptr.  This file sorts last so a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _inputs(graph, values, limbs, seed):
    import torch

    rng = np.random.default_rng(seed)
    X = rng.integers(0, 2 ** 64, size=(graph.n, values, limbs), dtype=np.uint64)
    rp = torch.from_numpy(graph.row_ptr).cuda()
    ci = torch.from_numpy(graph.col_idx).cuda()
    Xt = torch.from_numpy(X.view(np.int64)).cuda()
    return X, rp, ci, Xt


def test_noalloc_gather_matches_arena_gather_and_oracle_on_two_calls():
    import torch

    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    ctx = cc.Context(budget_bytes=1 << 30)
    stream = torch.cuda.current_stream().cuda_stream
    # call 1: more vertices, wider rows, many split tasks; call 2: smaller graph,
    # other widths and split, fewer tasks than call 1 left in the array
    cases = [(gg.rmat_graph(12, seed=3), 9, 2, 8), (gg.rmat_graph(10, seed=4), 5, 3, 4)]
    for i, (g, values, limbs, split) in enumerate(cases):
        assert np.diff(g.row_ptr).max() > split  # heavy vertices: the task path runs
        X, rp, ci, Xt = _inputs(g, values, limbs, seed=i)
        ref = torch.full_like(Xt, -1)
        out = torch.full_like(Xt, -1)
        ctx.table_gather(rp, ci, Xt, ref, values, limbs, split)
        cc.cc_table_gather_noalloc(rp, ci, Xt, out, values, limbs, split, stream=stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"call {i + 1} differs from cc_table_gather"
        expect = O.neighbour_sum(g, X, limbs)
        assert np.array_equal(out.cpu().numpy().view(np.uint64), expect), f"call {i + 1} differs from the oracle"
    ctx.close()


def test_noalloc_gather_allocates_nothing():
    import torch

    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    g = gg.rmat_graph(11, seed=6)
    X, rp, ci, Xt = _inputs(g, 6, 2, seed=7)
    out = torch.zeros_like(Xt)
    stream = torch.cuda.current_stream().cuda_stream
    cc.cc_table_gather_noalloc(rp, ci, Xt, out, 6, 2, 16, stream=stream)  # first call: address look-up
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        cc.cc_table_gather_noalloc(rp, ci, Xt, out, 6, 2, 16, stream=stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.array_equal(out.cpu().numpy().view(np.uint64), O.neighbour_sum(g, X, 2))


def test_noalloc_gather_rejects_bad_rows_and_inputs_beyond_its_scratch():
    import torch

    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    g = gg.rmat_graph(12, seed=5)
    # split 1: one task per neighbour of every vertex with two or more
    # neighbours, 32 KiB partial rows: far more than 64 MiB holds
    _, rp, ci, Xt = _inputs(g, 1000, 4, seed=9)
    out = torch.zeros_like(Xt)
    with pytest.raises(cc.CCError) as ei:
        cc.cc_table_gather_noalloc(rp, ci, Xt, out, 1000, 4, 1)
    assert ei.value.status == -11  # CC_ERR_CAPACITY
    ctx = cc.Context(budget_bytes=1 << 30)
    # a decreasing row_ptr (every neighbour id and row still in range): both
    # entry points refuse it before any gather runs
    bad_rp = torch.tensor([0, 3, 1, 4], dtype=torch.int64, device="cuda")
    bad_ci = torch.tensor([1, 2, 0, 1], dtype=torch.int32, device="cuda")
    bX = torch.zeros(3 * 2, dtype=torch.int64, device="cuda")
    bout = torch.zeros_like(bX)
    for call in (lambda: cc.cc_table_gather_noalloc(bad_rp, bad_ci, bX, bout, 2, 1, 1),
                 lambda: ctx.table_gather(bad_rp, bad_ci, bX, bout, 2, 1, 1)):
        with pytest.raises(cc.CCError) as ei:
            call()
        assert ei.value.status == -1  # CC_ERR_INVALID_ARG
    # a fitting call afterwards still agrees with the arena gather
    _, rp, ci, Xt = _inputs(g, 3, 1, seed=10)
    ref = torch.zeros_like(Xt)
    out = torch.zeros_like(Xt)
    ctx.table_gather(rp, ci, Xt, ref, 3, 1, 16)
    cc.cc_table_gather_noalloc(rp, ci, Xt, out, 3, 1, 16)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    ctx.close()
