"""Labelled templates: a counted map sends every template vertex to a graph
vertex with the same label (cc_template_load_labelled, cc_graph_set_labels).
Parity with the oracle's labelled counts, exact integers."""
import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def make_ctx(**kw):
    from paper_1804_09764_gb300 import cc

    return cc.Context(budget_bytes=kw.pop("budget_bytes", 3 << 30), **kw)


CASES = [("P5", 0, 3), ("caterpillar10", 2, 2), ("tree12", 1, 2)]


@pytest.mark.parametrize("cfg", [dict(), dict(split_threshold=12, batch=2, block_vertices=500, fused=0),
                                 dict(split_threshold=12, batch=2, block_vertices=500)])
def test_labelled_counts_match_oracle(cfg):
    g = gg.rmat_graph(10, seed=81)
    rng = np.random.default_rng(9)
    c = make_ctx(**cfg)
    gid = c.graph_load(g)
    for name, root, nlab in CASES:
        k, e = gg.template_edges(name)
        glab = rng.integers(0, nlab, g.n)
        tlab = rng.integers(0, nlab, k)
        c.graph_set_labels(gid, glab)
        tid = c.template_load(k, e, root, labels=tlab)
        res = c.count(gid, tid, seed=4, n_iter=2, want_maps=True)
        want = [O.count_maps(g, k, e, 0, seed=4, j=j, glabels=glab, tlabels=tlab) for j in range(2)]
        assert res["maps"] == want, name
        aut = O.automorphisms(k, e, tlab)
        assert res["aut"] == aut and res["counts"] == [m // aut for m in want]
    c.close()


def test_uniform_labels_equal_unlabelled():
    g = gg.rmat_graph(10, seed=82)
    k, e = gg.template_edges("tree12")
    c = make_ctx()
    gid = c.graph_load(g)
    c.graph_set_labels(gid, np.full(g.n, 7, dtype=np.uint8))
    plain = c.count(gid, c.template_load(k, e), seed=6, n_iter=3)
    lab = c.count(gid, c.template_load(k, e, labels=[7] * k), seed=6, n_iter=3)
    assert lab["counts"] == plain["counts"] and lab["aut"] == plain["aut"]
    c.close()


def test_labelled_single_vertex_and_errors():
    from paper_1804_09764_gb300 import cc

    g = gg.rmat_graph(8, seed=83)
    glab = np.arange(g.n) % 3
    c = make_ctx()
    gid = c.graph_load(g)
    t1 = c.template_load(1, np.zeros((0, 2), dtype=np.int32), labels=[2])
    tp = c.template_load(3, [(0, 1), (1, 2)], labels=[0, 1, 0])
    with pytest.raises(cc.CCError) as ei:
        c.count(gid, tp, seed=1, n_iter=1)  # no graph labels yet
    assert ei.value.status == -1
    c.graph_set_labels(gid, glab)
    assert c.count(gid, t1, seed=1, n_iter=2)["counts"] == [int((glab == 2).sum())] * 2
    want = O.count_maps(g, 3, [(0, 1), (1, 2)], 1, seed=1, j=0, glabels=glab, tlabels=[0, 1, 0])
    assert c.count(gid, tp, seed=1, n_iter=1, want_maps=True)["maps"] == [want]
    c.graph_set_labels(gid, None)
    with pytest.raises(cc.CCError):
        c.count(gid, tp, seed=1, n_iter=1)
    c.close()


def test_labelled_and_unlabelled_templates_in_one_merged_count():
    g = gg.rmat_graph(10, seed=84)
    glab = np.random.default_rng(2).integers(0, 2, g.n)
    k = 7
    trees = gg.all_trees(7)[:4]
    c = make_ctx()
    gid = c.graph_load(g)
    c.graph_set_labels(gid, glab)
    tids = [c.template_load(k, trees[0]), c.template_load(k, trees[1], labels=[0, 1, 0, 1, 0, 1, 0]),
            c.template_load(k, trees[2], labels=[1] * k), c.template_load(k, trees[3], labels=[0] * 6 + [1])]
    multi = c.count_multi(gid, tids, seed=8, n_iter=2)
    for tid, m in zip(tids, multi):
        assert m["counts"] == c.count(gid, tid, seed=8, n_iter=2)["counts"]
    c.close()


def test_labelled_requests_through_the_serving_loop():
    g = gg.rmat_graph(10, seed=85)
    glab = np.random.default_rng(4).integers(0, 3, g.n)
    c = make_ctx(max_slots=2)
    gid = c.graph_load(g)
    c.graph_set_labels(gid, glab)
    reqs = []
    for i, name in enumerate(["P5", "caterpillar10", "tree12"]):
        k, e = gg.template_edges(name)
        tid = c.template_load(k, e, labels=np.random.default_rng(10 + i).integers(0, 3, k))
        reqs.append((tid, c.submit(gid, tid, 20 + i, 3)))
    for i, (tid, rid) in enumerate(reqs):
        assert c.wait(rid, 3, timeout_s=120)["counts"] == c.count(gid, tid, seed=20 + i, n_iter=3)["counts"]
    c.close()
