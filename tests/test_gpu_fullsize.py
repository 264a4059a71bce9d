"""Parity at a benchmark workload's full size: R-MAT scale 20 (1,048,576
vertices), caterpillar-10 rooted at 2, 64 colourings, in the benchmark's
launch configuration.  Sampled per-vertex counts are checked one by one: a
map of T rooted at v stays within distance 2 of v (the template's depth from
its root), so the oracle on the induced 2-hop ball, with the original graph's
colours, gives the exact count at v."""
import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _ball(g, v, r):
    seen, frontier = {v}, [v]
    for _ in range(r):
        nxt = []
        for x in frontier:
            for u in g.col_idx[g.row_ptr[x]:g.row_ptr[x + 1]]:
                u = int(u)
                if u not in seen:
                    seen.add(u)
                    nxt.append(u)
        frontier = nxt
    return np.array(sorted(seen), dtype=np.int64)


def _induced(g, b):
    loc = {int(x): i for i, x in enumerate(b)}
    pairs = [(loc[int(x)], loc[int(u)]) for x in b for u in g.col_idx[g.row_ptr[x]:g.row_ptr[x + 1]]
             if int(u) in loc and loc[int(u)] > loc[int(x)]]
    return gg.csr_from_edges(b.size, np.array(pairs) if pairs else np.zeros((0, 2), dtype=np.int64)), loc


def test_rmat20_caterpillar10_sampled_vertices_at_full_size():
    from paper_1804_09764_gb300 import cc

    g = gg.rmat_graph(20, seed=20)
    k, e = gg.template_edges("caterpillar10")
    deg = np.diff(g.row_ptr)
    picked = []
    for v in np.random.default_rng(0).permutation(np.nonzero(deg >= 3)[0])[:20000]:
        b = _ball(g, int(v), 2)
        if 30 <= b.size <= 2000:
            picked.append((int(v), b))
        if len(picked) == 6:
            break
    c = cc.Context(budget_bytes=100 << 30)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 2)
    res = c.count(gid, tid, seed=12345, n_iter=64, sample_vertices=[v for v, _ in picked])
    nonzero = 0
    for j in (0, 37):
        for i, (v, b) in enumerate(picked):
            sg, loc = _induced(g, b)
            _, pv = O.count_maps(sg, k, e, 2, seed=12345, j=j, ids=b, per_vertex=True)
            assert res["samples"][j][i] == pv[loc[v]], (j, v)
            nonzero += pv[loc[v]] > 0
    assert nonzero >= 3
    c.close()
