"""Algorithm 1 end to end (cc_estimate): the median of group means equals the
one computed from the same colourings' exact counts, the estimate lands within
(1 +- epsilon) of closed-form copy numbers, and over-large samples are refused."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def make_ctx(**kw):
    from paper_1804_09764_gb300 import cc

    return cc.Context(budget_bytes=kw.pop("budget_bytes", 2 << 30), **kw)


def test_estimate_equals_median_of_means_of_plain_counts():
    from paper_1804_09764_gb300 import cc

    # P4 in K_12: C(12, 4) * 4! / |Aut| = 495 * 12 copies
    k, e = 4, [(0, 1), (1, 2), (2, 3)]
    copies = math.comb(12, 4) * math.factorial(4) // 2
    eps, delta, seed = 0.25, 0.1, 77
    n, t = cc.cc_iterations_for(k, eps, delta)
    c = make_ctx(batch=64)
    gid = c.graph_load(gg.complete_graph(12))
    tid = c.template_load(k, e)
    r = c.estimate(gid, tid, seed, eps, delta, first_iter=5)
    assert (r["n_iter"], r["groups"], r["per_group"]) == (n, t, n // t)
    plain = c.count(gid, tid, seed=seed, n_iter=n, first_iter=5)
    est = [x * (k ** k / math.factorial(k)) for x in plain["counts"]]
    assert r["estimate"] == pytest.approx(O.median_of_means(est, t), rel=1e-12)
    assert r["mean"] == pytest.approx(math.fsum(est) / n, rel=1e-12)
    assert r["min_group_mean"] <= r["estimate"] <= r["max_group_mean"]
    assert abs(r["estimate"] - copies) <= eps * copies
    c.close()


def test_estimate_on_the_template_itself():
    # G = T: one copy, the case where the variance bound is attained
    from paper_1804_09764_gb300 import cc

    k, e = gg.template_edges("P5")
    g = gg.csr_from_edges(k, e)
    c = make_ctx()
    gid = c.graph_load(g)
    tid = c.template_load(k, e)
    r = c.estimate(gid, tid, 3, 0.8, 0.1)
    assert r["n_iter"] == cc.cc_iterations_for(k, 0.8, 0.1)[0]
    assert abs(r["estimate"] - 1.0) <= 0.8
    c.close()


def test_estimate_refuses_samples_over_the_cap():
    from paper_1804_09764_gb300 import cc

    c = make_ctx()
    gid = c.graph_load(gg.complete_graph(8))
    tid = c.template_load(*gg.template_edges("P5"))
    with pytest.raises(cc.CCError) as ei:
        c.estimate(gid, tid, 1, 0.1, 0.01, max_iter=1000)
    assert ei.value.status == -11
    with pytest.raises(cc.CCError) as ei:
        c.estimate(gid, 999, 1, 0.5, 0.1)
    assert ei.value.status == -10
    c.close()
