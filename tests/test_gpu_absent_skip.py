"""Gathers that skip the entries a neighbour's row holds as zero by construction.

M(u, T, S) = 0 whenever col(u) is not in S, because the root of T is mapped to
u (Eq. 1, Section 2.1).  In a pass of one colouring the library's gathers load
only the entries of a neighbour's row whose colour set holds the neighbour's
colour (cc_options.full_rows = 0, the default).  These tests run the plan
shapes that reach every gather kernel taking the skip -- the fused chain and
select kernels, the column-segmented fused step with its leaf kernel, the
unfused warp-per-row gathers in each variant, the heavy-vertex tasks, one- and
multi-limb sources, sixteen colours -- at batch 1, with the skip and with whole
rows, and compare both with the oracle element by element."""
import functools

import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _count(g, k, e, root, seed, n_iter, **kw):
    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    c = cc.Context(budget_bytes=4 << 30, timing=1, batch=1, **kw)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, root)
    res = c.count(gid, tid, seed=seed, n_iter=n_iter, want_maps=True)
    inst = c.kernel_instances()
    c.close()
    launched = {name for kind in inst.values() for name in kind}
    return res, launched


def _check(g, k, e, root, seed, n_iter, **kw):
    maps = [O.count_maps(g, k, e, root, seed=seed, j=j) for j in range(n_iter)]
    for full_rows in (0, 1):
        res, launched = _count(g, k, e, root, seed, n_iter, full_rows=full_rows, **kw)
        assert res["maps"] == maps, f"full_rows={full_rows}"
        # the neighbour colours are written only when the gathers skip
        assert ("neighbour_colours_kernel" in launched) == (full_rows == 0)
    return launched


@functools.lru_cache(maxsize=None)
def _tree12_rmat10_maps():
    k, e = gg.template_edges("tree12")
    return O.count_maps(gg.rmat_graph(10, seed=2), k, e, 3, seed=9, j=0)


BROOM = [(0, 1), (1, 2), (2, 3)] + [(0, j) for j in range(4, 10)]


@pytest.mark.parametrize("fused", [0, 1])
def test_tree12_with_heavy_vertices_and_blocks(fused):
    # chain kernels, fused select, Algorithm 4 tasks (split 10), three blocks
    g = gg.rmat_graph(11, seed=44)
    k, e = gg.template_edges("tree12")
    launched = _check(g, k, e, 1, 17, 2, fused=fused, split_threshold=10, block_vertices=777)
    if fused:
        assert any(n.startswith("gather_select_chain_kernel") for n in launched)
    assert any(n.startswith("gather_tasks_kernel") for n in launched)


@pytest.mark.parametrize("chunks", [3, 64])
def test_column_segments(chunks):
    # segmented fused step + leaf kernel, segmented task gathers (gather_row_range)
    g = gg.rmat_graph(11, seed=46)
    launched = _check(g, 10, BROOM, 0, 23, 2, col_chunks=chunks, split_threshold=10, block_vertices=600)
    assert "leaf_chain_kernel<1>" in launched or "leaf_chain_kernel<2>" in launched


@pytest.mark.parametrize("mode", [4, 5, 6])
def test_unfused_gather_variants(mode):
    # warp-per-row gathers: whole-row L2 prefetch (4), one pass without a
    # counter (5), two rows in flight (6)
    g = gg.rmat_graph(11, seed=45)
    _check(g, 10, BROOM, 0, 19, 2, fused=0, gather_mode=mode, split_threshold=10, block_vertices=700)


@pytest.mark.parametrize("width", [128, 256])
@pytest.mark.parametrize("fused", [0, 1])
def test_multi_limb_sources(width, fused):
    # every table at two or four limbs: the limb-wise neighbour sums (residues
    # mod 2^width), heavy vertices on the task path
    g = gg.rmat_graph(10, seed=2)
    k, e = gg.template_edges("tree12")
    m = _tree12_rmat10_maps()
    for full_rows in (0, 1):
        res, launched = _count(g, k, e, 3, 9, 1, full_rows=full_rows, width_bits=width, fused=fused,
                               split_threshold=10)
        assert res["exact"] == 0 and res["limbs"] == width // 64
        assert res["counts"][0] == m % (1 << width), f"full_rows={full_rows}"
        assert ("neighbour_colours_kernel" in launched) == (full_rows == 0)


def test_sixteen_colours():
    # k = 16: colour 15 travels in the top bits of the broadcast id
    g = gg.disjoint_union(gg.er_graph(300, 6, seed=5), gg.star_graph(40))
    e = gg.prufer_tree(16, seed=4)
    _check(g, 16, e, 0, 9, 1, split_threshold=16)


def test_cuda_graph_replay_and_autotuner():
    # the pass captured once and replayed for every colouring: the neighbour
    # colours are rewritten inside the replay; the autotuner times every
    # gather variant (those that read whole rows and those that skip)
    g = gg.rmat_graph(11, seed=47)
    k, e = gg.template_edges("tree12")
    _check(g, k, e, 1, 31, 3, use_cuda_graph=1, autotune=1, split_threshold=40)
