"""The allocation-free table gather against the allocating one, through the C ABI.

cc_table_gather_noalloc exists for callers that cannot allocate device memory
(a framework that owns all of it through its own pool, a latency-bound loop
where cudaMalloc/cudaFree are not acceptable, a fixed memory budget).  It keeps
its scratch in a fixed file-scope device array instead of the context arena.
These checks run it twice in a row on different inputs (so the second call
would see anything the first left behind in the shared array) and compare each
result bit for bit with cc_table_gather on the same inputs; integer sums have
no tolerance.  This file sorts last so a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _device_inputs(graph, values, limbs, seed):
    import torch

    rng = np.random.default_rng(seed)
    X = rng.integers(0, 2 ** 64, size=(graph.n, values, limbs), dtype=np.uint64)
    rp = torch.from_numpy(graph.row_ptr).cuda()
    ci = torch.from_numpy(graph.col_idx).cuda()
    Xt = torch.from_numpy(X.view(np.int64)).cuda()
    return rp, ci, Xt


def test_noalloc_gather_matches_arena_gather_on_two_calls():
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
        rp, ci, Xt = _device_inputs(g, values, limbs, seed=i)
        ref = torch.full_like(Xt, -1)
        out = torch.full_like(Xt, -1)
        ctx.table_gather(rp, ci, Xt, ref, values, limbs, split)
        cc.cc_table_gather_noalloc(rp, ci, Xt, out, values, limbs, split, stream=stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"call {i + 1} differs from cc_table_gather"
    ctx.close()


def test_noalloc_gather_rejects_inputs_beyond_its_scratch():
    import torch

    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    g = gg.rmat_graph(12, seed=5)
    # split 1: one task per neighbour of every vertex with two or more
    # neighbours, 32 KiB partial rows: far more than 64 MiB holds
    rp, ci, Xt = _device_inputs(g, 1000, 4, seed=9)
    out = torch.zeros_like(Xt)
    with pytest.raises(cc.CCError) as ei:
        cc.cc_table_gather_noalloc(rp, ci, Xt, out, 1000, 4, 1)
    assert ei.value.status == -11  # CC_ERR_CAPACITY
    # a fitting call afterwards still agrees with the arena gather
    ctx = cc.Context(budget_bytes=1 << 30)
    rp, ci, Xt = _device_inputs(g, 3, 1, seed=10)
    ref = torch.zeros_like(Xt)
    out = torch.zeros_like(Xt)
    ctx.table_gather(rp, ci, Xt, ref, 3, 1, 16)
    cc.cc_table_gather_noalloc(rp, ci, Xt, out, 3, 1, 16)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    ctx.close()
