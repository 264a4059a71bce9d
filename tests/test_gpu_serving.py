"""Continuous-batching serving loop: results in the mix equal results alone.

Requests over several resident graphs and templates are submitted while others
are running; every result must be bit-identical to the same count run alone
through cc_count (exact integers: the tolerance is zero) and, for a sample, to
the oracle.  Requests on one graph with isomorphic templates share passes:
one launch carries colourings of both.  Also: cancellation, unknown handles,
and the latency statistics.
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def make_ctx(**kw):
    from paper_1804_09764_gb300 import cc

    return cc.Context(budget_bytes=kw.pop("budget_bytes", 6 << 30), **kw)


def test_mix_equals_alone():
    rng = np.random.default_rng(42)
    graphs = [gg.rmat_graph(10, seed=1), gg.rmat_graph(11, seed=2), gg.er_graph(3000, 8, seed=3)]
    c = make_ctx(max_slots=3, batch=4)
    gids = [c.graph_load(g) for g in graphs]
    reqs = []
    for i in range(14):
        k = int(rng.integers(3, 10))
        e = gg.prufer_tree(k, 500 + i)
        gi = int(rng.integers(0, len(graphs)))
        reqs.append(dict(g=gi, k=k, e=e, tid=c.template_load(k, e), seed=int(rng.integers(0, 2 ** 40)),
                         n_iter=int(rng.integers(1, 7)), first=int(rng.integers(0, 100))))
    # alone
    for r in reqs:
        r["alone"] = c.count(gids[r["g"]], r["tid"], seed=r["seed"], n_iter=r["n_iter"], first_iter=r["first"])
    # in the mix: half up front, the rest while the first ones run
    ids = []
    for r in reqs[:7]:
        ids.append(c.submit(gids[r["g"]], r["tid"], r["seed"], r["n_iter"], r["first"]))
    time.sleep(0.01)
    for r in reqs[7:]:
        ids.append(c.submit(gids[r["g"]], r["tid"], r["seed"], r["n_iter"], r["first"]))
    for rid, r in zip(ids, reqs):
        res = c.wait(rid, r["n_iter"], timeout_s=120)
        assert res["counts"] == r["alone"]["counts"]
        assert res["estimate"] == r["alone"]["estimate"]
    st = c.serve_stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["p50_latency_s"] <= st["p99_latency_s"]
    # oracle spot check of two requests
    for r in reqs[:2]:
        g = graphs[r["g"]]
        aut = O.automorphisms(r["k"], r["e"])
        want = [O.count_maps(g, r["k"], r["e"], 0, seed=r["seed"], j=r["first"] + j) // aut
                for j in range(r["n_iter"])]
        assert r["alone"]["counts"] == want
    c.close()


def test_cancel_and_errors():
    from paper_1804_09764_gb300 import cc

    c = make_ctx(max_slots=1)
    gid = c.graph_load(gg.rmat_graph(12, seed=7))
    tid = c.template_load(*gg.template_edges("tree12"))
    tid2 = c.template_load(*gg.template_edges("P5"))
    r1 = c.submit(gid, tid, 1, 8)
    r2 = c.submit(gid, tid2, 2, 8)   # another template class: queued behind r1 (one slot)
    c.cancel(r2)
    with pytest.raises(cc.CCError) as ei:
        c.wait(r2, 8, timeout_s=120)
    assert ei.value.status == -9
    res = c.wait(r1, 8, timeout_s=120)
    assert len(res["counts"]) == 8
    with pytest.raises(cc.CCError) as ei:
        c.poll(12345, 1)
    assert ei.value.status == -10
    with pytest.raises(cc.CCError) as ei:
        c.submit(gid, 999, 1, 1)
    assert ei.value.status == -10
    c.close()


def test_one_launch_carries_two_requests():
    # two isomorphic templates (the second relabelled and rooted elsewhere) on
    # one graph: one group, and passes whose colourings belong to both requests
    k = 7
    e1 = gg.prufer_tree(k, 4242)
    perm = [3, 6, 0, 5, 1, 4, 2]
    e2 = [(perm[a], perm[b]) for a, b in e1]
    g = gg.rmat_graph(11, seed=9)
    c = make_ctx(max_slots=1, batch=16)
    gid = c.graph_load(g)
    t1, t2 = c.template_load(k, e1, 0), c.template_load(k, e2, perm[3])
    alone1 = c.count(gid, t1, seed=11, n_iter=40, first_iter=7)
    alone2 = c.count(gid, t2, seed=12, n_iter=6, first_iter=3)
    r1 = c.submit(gid, t1, 11, 40, 7)
    r2 = c.submit(gid, t2, 12, 6, 3)
    got1 = c.wait(r1, 40, timeout_s=120)
    got2 = c.wait(r2, 6, timeout_s=120)
    assert got1["counts"] == alone1["counts"] and got2["counts"] == alone2["counts"]
    st = c.serve_stats()
    assert st["shared_passes"] >= 1, st
    assert st["colourings_run"] == 46 and st["passes"] == 3, st  # one after the other: 3 + 1 passes
    aut = O.automorphisms(k, e2)
    assert got2["counts"][0] == O.count_maps(g, k, e2, 0, seed=12, j=3) // aut
    c.close()


def test_served_group_replans_to_a_batch_that_fits():
    # batch=16 pins the number of colourings a plan takes, and a pass of all
    # six colourings does not fit this arena: cc_count refuses the count, while
    # the serving loop re-plans its group with half as many colourings per
    # pass until the workspace fits; the counts are those of the count alone
    from paper_1804_09764_gb300 import cc

    g = gg.rmat_graph(12, seed=13)
    k, e = gg.template_edges("tree12")
    big = make_ctx(batch=1)
    gid = big.graph_load(g)
    tid = big.template_load(k, e, 1)
    ws1 = big.plan_info(gid, tid)["workspace_bytes"]
    alone = big.count(gid, tid, seed=31, n_iter=6)["counts"]
    big.close()
    c = make_ctx(batch=16, budget_bytes=int(3.5 * ws1) + (96 << 20))
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 1)
    with pytest.raises(cc.CCError) as ei:
        c.count(gid, tid, seed=31, n_iter=6)
    assert ei.value.status == -5  # CC_ERR_BUDGET
    r = c.submit(gid, tid, 31, 6)
    assert c.wait(r, 6, timeout_s=120)["counts"] == alone
    st = c.serve_stats()
    assert st["completed"] == 1 and st["colourings_run"] == 6 and st["passes"] >= 2, st
    c.close()
