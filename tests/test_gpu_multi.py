"""Several templates over the same colourings (cc_count_multi): every result
equals the template counted alone (exact integers, tolerance zero) and the
oracle; rooted subtrees shared between templates are planned once."""
import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def make_ctx(**kw):
    from paper_1804_09764_gb300 import cc

    return cc.Context(budget_bytes=kw.pop("budget_bytes", 3 << 30), **kw)


def _load(c, tmpls):
    return [c.template_load(k, e, r) for k, e, r in tmpls]


@pytest.mark.parametrize("cfg", [dict(), dict(split_threshold=12, batch=2, block_vertices=500)])
def test_multi_equals_alone_and_oracle(cfg):
    g = gg.rmat_graph(10, seed=71)
    k = 7
    tmpls = [(k, gg.prufer_tree(k, 900 + i), -1) for i in range(5)]
    tmpls.append(tmpls[0])                                   # the same template twice
    tmpls.append((k, tmpls[1][1], 0))                        # the same tree, another root
    c = make_ctx(**cfg)
    gid = c.graph_load(g)
    tids = _load(c, tmpls)
    multi = c.count_multi(gid, tids, seed=5, n_iter=3, first_iter=2, want_maps=True)
    for tid, m in zip(tids, multi):
        alone = c.count(gid, tid, seed=5, n_iter=3, first_iter=2, want_maps=True)
        assert m["counts"] == alone["counts"] and m["maps"] == alone["maps"]
        assert m["estimate"] == alone["estimate"] and m["aut"] == alone["aut"]
    for (kk, e, r), m in list(zip(tmpls, multi))[:2]:
        want = [O.count_maps(g, kk, e, 0, seed=5, j=2 + j) for j in range(3)]
        assert m["maps"] == want
    info = c.multi_plan_info(gid, tids)
    assert info["chains"] < info["chains_separate"]
    assert info["updates_per_colouring"] < info["updates_per_colouring_separate"]
    c.close()


def test_multi_with_different_root_widths():
    # K_{1,7} on a star with 1500 leaves needs two limbs; P8 fits in one: the
    # merged plan runs both roots at two limbs and keeps P8's low limb
    g = gg.star_graph(1500)
    star = [(0, j) for j in range(1, 8)]
    path = [(j, j + 1) for j in range(7)]
    c = make_ctx()
    gid = c.graph_load(g)
    tids = [c.template_load(8, star, 0), c.template_load(8, path)]
    multi = c.count_multi(gid, tids, seed=9, n_iter=2, want_maps=True)
    for tid, m in zip(tids, multi):
        alone = c.count(gid, tid, seed=9, n_iter=2, want_maps=True)
        assert m["counts"] == alone["counts"] and m["limbs"] == alone["limbs"]
    assert multi[0]["limbs"] == 2 and multi[1]["limbs"] == 1
    assert multi[0]["maps"] == [O.count_maps(g, 8, star, 0, seed=9, j=j) for j in range(2)]
    assert multi[1]["counts"] == [0, 0]
    c.close()


def test_multi_errors_and_trivial_cases():
    from paper_1804_09764_gb300 import cc

    c = make_ctx()
    gid = c.graph_load(gg.rmat_graph(8, seed=3))
    t5 = c.template_load(*gg.template_edges("P5"))
    t3 = c.template_load(3, [(0, 1), (1, 2)])
    for tids, status in [([t5, t3], -1), ([t5, 999], -10), ([], -1)]:
        with pytest.raises(cc.CCError) as ei:
            c.count_multi(gid, tids, seed=1, n_iter=1)
        assert ei.value.status == status
    t1 = c.template_load(1, np.zeros((0, 2), dtype=np.int32))
    res = c.count_multi(gid, [t1, t1], seed=1, n_iter=2)
    assert res[0]["counts"] == res[1]["counts"] == c.count(gid, t1, seed=1, n_iter=2)["counts"]
    res = c.count_multi(gid, [t5], seed=1, n_iter=0)
    assert res[0]["counts"] == []
    c.close()
