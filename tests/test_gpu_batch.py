"""Graph batches: many graphs resident as one disjoint union, every DP launch
covering all of them (cc_graph_load_batch, cc_count_batch), against the oracle.

Eq. 1 is local to a vertex's neighbourhood, so the tables of a disjoint union
are the tables of its parts, and the root sum of Eq. 3 split by member graph
gives each member's colourful maps.  A member's colours are drawn from its own
vertex ids, so its counts must equal the oracle's for that graph alone, bit
for bit, whatever else shares the launch.  The members below mix sizes and
shapes (an all-isolated graph, a cycle, a star, R-MAT and Erdos-Renyi graphs),
and the runs cross vertex blocks in the middle of members and take several
colouring passes with a ragged last one."""
import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def members():
    return [gg.er_graph(300, 6, seed=1), gg.rmat_graph(9, seed=2), gg.csr_from_edges(7, []),
            gg.cycle_graph(12), gg.star_graph(20), gg.er_graph(1000, 8, seed=3), gg.rmat_graph(8, seed=5)]


def make_ctx(**kw):
    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    return cc.Context(budget_bytes=kw.pop("budget_bytes", 2 << 30), **kw)


@pytest.mark.parametrize("opts", [dict(batch=2), dict(batch=1, block_vertices=700), dict(batch=3, fused=0)])
def test_batch_counts_equal_each_graph_alone_and_the_oracle(opts):
    gs = members()
    k, e = 6, gg.prufer_tree(6, 606)
    seed, n_iter = 8080, 3
    aut = O.automorphisms(k, e)
    ctx = make_ctx(**opts)
    gid = ctx.graph_load_batch(gs)
    assert ctx.graph_members(gid) == len(gs)
    tid = ctx.template_load(k, e, 0)
    res = ctx.count_batch(gid, tid, seed=seed, n_iter=n_iter, want_maps=True)
    whole = ctx.count(gid, tid, seed=seed, n_iter=n_iter)
    est_sum = 0.0
    for i, g in enumerate(gs):
        maps = [O.count_maps(g, k, e, 0, seed=seed, j=j) for j in range(n_iter)]
        assert res["maps"][i] == maps, f"member {i}"
        assert res["counts"][i] == [O.copies_from_maps(m, aut) for m in maps], f"member {i}"
        ests = [O.estimate(O.copies_from_maps(m, aut), k) for m in maps]
        assert res["estimates"][i] == pytest.approx(sum(ests) / n_iter, rel=1e-12, abs=0)
        est_sum += res["estimates"][i]
        # the member loaded on its own
        alone = ctx.graph_load(g)
        assert ctx.count(alone, tid, seed=seed, n_iter=n_iter)["counts"] == res["counts"][i]
        ctx.graph_free(alone)
    # the batch as one graph: the sums over its members
    assert whole["counts"] == [sum(res["counts"][i][j] for i in range(len(gs))) for j in range(n_iter)]
    assert res["estimate"] == pytest.approx(est_sum, rel=1e-12)
    ctx.close()


def test_batch_trivial_templates_and_refusals():
    from paper_1804_09764_gb300 import cc

    gs = members()
    ctx = make_ctx()
    gid = ctx.graph_load_batch(gs)
    # k = 1: every vertex of each member, isolated ones included
    t1 = ctx.template_load(1, [])
    r = ctx.count_batch(gid, t1, seed=1, n_iter=2)
    assert r["counts"] == [[g.n, g.n] for g in gs]
    # k = 2: each member's colourful edges under its own colourings
    t2 = ctx.template_load(2, [(0, 1)])
    r = ctx.count_batch(gid, t2, seed=3, n_iter=2)
    for i, g in enumerate(gs):
        assert r["counts"][i] == [O.count_maps(g, 2, [(0, 1)], 0, seed=3, j=j) // 2 for j in range(2)]
    # an edge joining two members is refused, and so are decreasing offsets
    u = gg.csr_from_edges(11, [(i, (i + 1) % 5) for i in range(5)] + [(5 + i, 5 + (i + 1) % 6) for i in range(6)]
                          + [(4, 5)])
    with pytest.raises(cc.CCError) as ei:
        ctx.graph_load_batch_csr([0, 5, 11], u.row_ptr, u.col_idx)
    assert ei.value.status == -2  # CC_ERR_BAD_GRAPH
    with pytest.raises(cc.CCError) as ei:
        ctx.graph_load_batch_csr([0, 6, 5, 11], u.row_ptr, u.col_idx)
    assert ei.value.status == -1  # CC_ERR_INVALID_ARG
    # without the joining edge the same two cycles load
    v = gg.csr_from_edges(11, [(i, (i + 1) % 5) for i in range(5)] + [(5 + i, 5 + (i + 1) % 6) for i in range(6)])
    g2 = ctx.graph_load_batch_csr([0, 5, 11], v.row_ptr, v.col_idx, validate=True)
    tc = ctx.template_load(3, [(0, 1), (1, 2)])
    r = ctx.count_batch(g2, tc, seed=9, n_iter=1)
    cyc = [gg.cycle_graph(5), gg.cycle_graph(6)]
    assert r["counts"] == [[O.count_maps(c, 3, [(0, 1), (1, 2)], 0, seed=9, j=0) // 2] for c in cyc]
    ctx.close()
