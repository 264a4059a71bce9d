"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element
by element, on the same seeded inputs.  Integer counts must be bit-exact; the
FP64 estimate must agree to a relative 1e-12.

Sizes are chosen so the oracle finishes in seconds while the GPU path still
crosses several vertex blocks with a ragged tail, splits heavy neighbour lists
into tasks, and runs several colouring passes with a ragged last pass."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

EST_RTOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    c = cc.Context(budget_bytes=8 << 30)
    yield c
    c.close()


def make_ctx(**kw):
    from paper_1804_09764_gb300 import cc

    return cc.Context(budget_bytes=kw.pop("budget_bytes", 4 << 30), **kw)


def oracle_maps(g, k, e, root, seed, js):
    return [O.count_maps(g, k, e, root, seed=seed, j=j) for j in js]


def check_counts(res, maps, k, aut, limbs):
    M = 1 << (64 * limbs)
    for j, m in enumerate(maps):
        if res["exact"]:
            assert res["counts"][j] == m // aut, f"colouring {j}"
            assert m % aut == 0
        else:
            assert res["counts"][j] == m % M, f"colouring {j}"
    if res["exact"] and maps:
        est = [O.estimate(m // aut, k) for m in maps]
        mean = math.fsum(est) / len(est)
        assert res["estimate"] == pytest.approx(mean, rel=EST_RTOL, abs=1e-300)


# ------------------------------------------------------------------ workload 1

def test_er2000_p5_one_colouring(ctx):
    # ER n=2000, d=8; P5; k=5; one colouring (the tiny plain-method workload)
    g = gg.er_graph(2000, 8, seed=1)
    k, e = gg.template_edges("P5")
    gid = ctx.graph_load(g, validate=True)
    for root in range(k):
        tid = ctx.template_load(k, e, root)
        res = ctx.count(gid, tid, seed=1, n_iter=1, want_maps=True)
        maps = oracle_maps(g, k, e, root, 1, [0])
        assert res["maps"] == maps
        check_counts(res, maps, k, 2, res["limbs"])
        ctx.template_free(tid)
    ctx.graph_free(gid)


# ------------------------------------------------------------------ R-MAT, several templates

@pytest.mark.parametrize("name,scale,root,n_iter", [
    ("caterpillar10", 11, 2, 5),
    ("tree12", 10, 3, 2),
    ("spider15", 9, 0, 1),
])
def test_rmat_templates_blocks_splits_batches(name, scale, root, n_iter):
    g = gg.rmat_graph(scale, seed=scale)
    k, e = gg.template_edges(name)
    aut = O.automorphisms(k, e)
    maps = oracle_maps(g, k, e, root, 7, range(n_iter))
    # several tiles: 3 vertex blocks with a ragged tail, heavy lists split in tasks of 16,
    # batches of 2 colourings with a ragged last pass
    for kw in (dict(), dict(block_vertices=701, split_threshold=16, batch=2)):
        c = make_ctx(**kw)
        gid = c.graph_load(g)
        tid = c.template_load(k, e, root)
        res = c.count(gid, tid, seed=7, n_iter=n_iter, want_maps=True)
        assert res["maps"] == [m % (1 << (64 * res["limbs"])) for m in maps]
        check_counts(res, maps, k, aut, res["limbs"])
        c.close()


def test_partition_invariance_and_planner_root():
    g = gg.rmat_graph(10, seed=5)
    k, e = gg.template_edges("caterpillar10")
    c = make_ctx(split_threshold=32)
    gid = c.graph_load(g)
    ref = O.count_maps(g, k, e, 0, seed=3, j=4)
    for root in list(range(k)) + [-1]:
        tid = c.template_load(k, e, root)
        res = c.count(gid, tid, seed=3, n_iter=1, first_iter=4, want_maps=True)
        assert res["maps"][0] == ref
        c.template_free(tid)
    c.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_trees(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(3, 10))
    e = gg.prufer_tree(k, 77 + seed)
    g = gg.rmat_graph(9, seed=100 + seed) if seed % 2 else gg.er_graph(700, 6, seed=seed)
    root = int(rng.integers(0, k))
    c = make_ctx(batch=3, split_threshold=24)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, root)
    res = c.count(gid, tid, seed=seed, n_iter=4, want_maps=True)
    maps = oracle_maps(g, k, e, root, seed, range(4))
    check_counts(res, maps, k, O.automorphisms(k, e), res["limbs"])
    c.close()


# ------------------------------------------------------------------ integer widths

@pytest.mark.parametrize("width", [64, 128, 192, 256])
def test_forced_width_residues(width):
    g = gg.rmat_graph(10, seed=2)
    k, e = gg.template_edges("tree12")
    c = make_ctx(width_bits=width)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 3)
    res = c.count(gid, tid, seed=9, n_iter=1)
    m = O.count_maps(g, k, e, 3, seed=9, j=0)
    assert res["exact"] == 0 and res["limbs"] == width // 64
    assert res["counts"][0] == m % (1 << width)
    c.close()


def test_wide_exact_counts_star_on_star():
    # counts above 2^128: star template on K_{1,4000}, k = 14
    k = 14
    e = [(0, i) for i in range(1, k)]
    g = gg.star_graph(4000)
    c = make_ctx(split_threshold=64)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 0)
    res = c.count(gid, tid, seed=5, n_iter=2, want_maps=True)
    maps = oracle_maps(g, k, e, 0, 5, range(2))
    assert res["limbs"] >= 3
    assert res["maps"] == maps
    assert max(maps).bit_length() > 128
    c.close()


def test_more_launches_than_work_counters():
    # one-vertex blocks: the root chain (root 2) gathers the shared table of
    # the two 4-vertex stars twice, one persistent launch per block each, so
    # one pass takes more than twice as many persistent launches as there are
    # blocks -- far more than the 4096 work counters the pass clears at its
    # start; the counters are cleared again (in stream order) when used up,
    # and the counts stay exact
    g = gg.rmat_graph(12, seed=21)
    k, e = gg.template_edges("caterpillar10")
    c = make_ctx(block_vertices=1, batch=1, split_threshold=16)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 2)
    info = c.plan_info(gid, tid)
    assert info["n_blocks"] > 2048
    res = c.count(gid, tid, seed=6, n_iter=1, want_maps=True)
    assert res["maps"] == oracle_maps(g, k, e, 2, 6, range(1))
    c.close()


# ------------------------------------------------------------------ per-vertex outputs

def test_sampled_vertices_match_oracle_per_vertex():
    g = gg.rmat_graph(10, seed=8)
    k, e = gg.template_edges("caterpillar10")
    _, pv = O.count_maps(g, k, e, 2, seed=4, j=1, per_vertex=True)
    c = make_ctx(block_vertices=333, split_threshold=20)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 2)
    sample = list(range(0, g.n, 7)) + [g.n - 1]
    res = c.count(gid, tid, seed=4, n_iter=1, first_iter=1, sample_vertices=sample)
    assert res["samples"][0] == [pv[v] for v in sample]
    c.close()


# ------------------------------------------------------------------ edge cases

def test_edge_cases():
    c = make_ctx()
    # empty graph and graph without edges
    for g in (gg.csr_from_edges(0, np.zeros((0, 2))), gg.csr_from_edges(5, np.zeros((0, 2)))):
        gid = c.graph_load(g)
        for k, e in ((1, []), (2, [(0, 1)]), (4, [(0, 1), (1, 2), (2, 3)])):
            tid = c.template_load(k, e)
            res = c.count(gid, tid, seed=1, n_iter=2)
            assert res["counts"] == [g.n if k == 1 else 0] * 2
        c.graph_free(gid)
    # k = 1 counts every vertex, isolated ones included; k = 2 counts colourful edges
    g = gg.csr_from_edges(10, [(0, 1), (1, 2), (5, 6)])
    gid = c.graph_load(g)
    tid = c.template_load(1, [])
    assert c.count(gid, tid, seed=1, n_iter=1)["counts"] == [10]
    tid = c.template_load(2, [(0, 1)])
    res = c.count(gid, tid, seed=11, n_iter=3)
    assert res["counts"] == [O.count_maps(g, 2, [(0, 1)], 0, seed=11, j=j) // 2 for j in range(3)]
    # template larger than any component: zero
    tid = c.template_load(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    assert c.count(gid, tid, seed=1, n_iter=1)["counts"] == [0]
    c.close()


def test_bad_inputs_raise():
    from paper_1804_09764_gb300 import cc

    c = make_ctx()
    rp = np.array([0, 1, 1], dtype=np.int64)
    with pytest.raises(cc.CCError) as ei:   # asymmetric
        c.graph_load_csr(rp, np.array([1], dtype=np.int32), validate=True)
    assert ei.value.status == -2
    with pytest.raises(cc.CCError) as ei:   # self-loop
        c.graph_load_csr(np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), validate=True)
    assert ei.value.status == -2
    with pytest.raises(cc.CCError) as ei:   # not a tree
        c.template_load(3, [(0, 1), (1, 0)])
    assert ei.value.status == -3
    g = gg.er_graph(100, 4, seed=1)
    gid = c.graph_load(g)
    tid = c.template_load(5, gg.template_edges("P5")[1])
    with pytest.raises(cc.CCError) as ei:   # capacity
        c.count(gid, tid, seed=1, n_iter=1, limbs_capacity=0)
    c.close()


def test_budget_refusal():
    from paper_1804_09764_gb300 import cc

    g = gg.rmat_graph(12, seed=1)
    c = make_ctx(budget_bytes=8 << 20)
    gid = c.graph_load(g)
    tid = c.template_load(*gg.template_edges("tree12"), 3)
    with pytest.raises(cc.CCError) as ei:
        c.count(gid, tid, seed=1, n_iter=1)
    assert ei.value.status == -5
    c.close()


# ------------------------------------------------------------------ table gather on its own

@pytest.mark.parametrize("limbs,split", [(1, 0), (2, 8), (3, 5), (4, 16)])
def test_table_gather_matches_oracle_neighbour_sum(limbs, split):
    import torch

    g = gg.rmat_graph(9, seed=31)
    values = 7
    rng = np.random.default_rng(limbs)
    X = rng.integers(0, 2 ** 64, size=(g.n, values, limbs), dtype=np.uint64)
    expect = O.neighbour_sum(g, X, limbs)
    c = make_ctx()
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    Xt = torch.from_numpy(X.view(np.int64)).cuda()
    A = torch.full_like(Xt, -1)
    c.table_gather(rp, ci, Xt, A, values, limbs, split)
    assert np.array_equal(A.cpu().numpy().view(np.uint64), expect)
    c.close()


def test_bulk_and_warp_gathers_agree_with_oracle():
    # gather_mode 0: bulk-copy (TMA) gather for rows of >= 1 KiB; 1: scalar warp
    # gather; 2: vectorised warp gather; 3: group gather; 4: warp gather + L2 prefetch
    g = gg.rmat_graph(11, seed=21)
    k, e = gg.template_edges("tree12")
    maps = oracle_maps(g, k, e, 1, 13, range(3))
    for mode in (0, 1, 2, 3, 4, 5):
        c = make_ctx(gather_mode=mode, split_threshold=12, batch=2, block_vertices=900)
        gid = c.graph_load(g)
        tid = c.template_load(k, e, 1)
        res = c.count(gid, tid, seed=13, n_iter=3, want_maps=True)
        assert res["maps"] == maps, f"gather_mode {mode}"
        c.close()


def test_cuda_graph_replay_and_plan_cache():
    # the per-pass schedule captured once as a CUDA graph and replayed for every
    # pass and every later call with the same plan
    g = gg.rmat_graph(10, seed=12)
    k, e = gg.template_edges("caterpillar10")
    c = make_ctx(use_cuda_graph=1, batch=2, split_threshold=16)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 2)
    for first in (0, 5):
        res = c.count(gid, tid, seed=21, n_iter=3, first_iter=first, want_maps=True)
        assert res["maps"] == oracle_maps(g, k, e, 2, 21, range(first, first + 3))
    c.close()


def test_autotuned_plan_matches_oracle():
    # the first pass times every gather variant per site; all passes must stay exact
    g = gg.rmat_graph(11, seed=33)
    k, e = gg.template_edges("tree12")
    c = make_ctx(autotune=1, use_cuda_graph=1, batch=2, split_threshold=40)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 1)
    for first in (0, 4):
        res = c.count(gid, tid, seed=5, n_iter=4, first_iter=first, want_maps=True)
        assert res["maps"] == oracle_maps(g, k, e, 1, 5, range(first, first + 4))
    c.close()


def test_autotuned_split_threshold_matches_oracle():
    # with split_threshold, col_chunks and block_vertices at 0 the first count
    # times candidate shapes (task size, column segments, block size) and keeps
    # the fastest; the counts stay exact and later plans use it
    g = gg.rmat_graph(12, seed=34)
    assert np.diff(g.row_ptr).max() > 1024
    k, e = gg.template_edges("tree12")
    c = make_ctx(autotune=1, batch=2)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 1)
    res = c.count(gid, tid, seed=7, n_iter=2, want_maps=True)
    assert res["maps"] == oracle_maps(g, k, e, 1, 7, range(2))
    info = c.plan_info(gid, tid)
    assert info["split_threshold"] in (1024, 4096, 16384)
    assert info["col_chunks"] in (0, 1, 4, 16) and info["shape_tuned"] == 1
    res = c.count(gid, tid, seed=7, n_iter=2, first_iter=2, want_maps=True)
    assert res["maps"] == oracle_maps(g, k, e, 1, 7, range(2, 4))
    c.close()


@pytest.mark.parametrize("fused", [0, 1])
def test_fused_and_unfused_gather_select(fused):
    # a = 1 steps: fused gather + select kernel against the separate kernels, with
    # heavy vertices (split 10), vertex blocks and batches
    g = gg.rmat_graph(11, seed=44)
    k, e = gg.template_edges("tree12")
    maps = oracle_maps(g, k, e, 1, 17, range(3))
    c = make_ctx(fused=fused, split_threshold=10, batch=2, block_vertices=777)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 1)
    res = c.count(gid, tid, seed=17, n_iter=3, want_maps=True)
    assert res["maps"] == maps
    c.close()


@pytest.mark.parametrize("fused", [0, 1])
def test_leaf_chain_after_fused_step(fused):
    # broom: hub 0 with the path 1-2-3 and six leaves.  The hub's chain is one
    # a = 1 step (the path) followed by six p = 1 steps whose rows widen and then
    # narrow (C(10, h) for h = 4..10), run as one kernel per block when fused;
    # heavy vertices (split 10), three vertex blocks and two colourings per pass.
    g = gg.rmat_graph(11, seed=45)
    k = 10
    e = np.array([(0, 1), (1, 2), (2, 3)] + [(0, j) for j in range(4, 10)], dtype=np.int32)
    maps = oracle_maps(g, k, e, 0, 19, range(3))
    c = make_ctx(fused=fused, split_threshold=10, batch=2, block_vertices=600)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 0)
    res = c.count(gid, tid, seed=19, n_iter=3, want_maps=True)
    assert res["maps"] == maps
    c.close()


@pytest.mark.parametrize("chunks", [1, 2, 3, 7, 64])
@pytest.mark.parametrize("fused", [0, 1])
def test_column_segments(chunks, fused):
    # rows split into `chunks` column segments, run segment-major (64: more
    # segments than warp sweeps, so trailing segments are empty); chains of leaf
    # steps after a fused step take the separate leaf kernel when chunks > 1
    g = gg.rmat_graph(11, seed=46)
    k = 10
    broom = [(0, 1), (1, 2), (2, 3)] + [(0, j) for j in range(4, 10)]
    cat = gg.template_edges("caterpillar10")[1]
    c = make_ctx(col_chunks=chunks, fused=fused, split_threshold=10, batch=2, block_vertices=600)
    gid = c.graph_load(g)
    for e, root in [(broom, 0), (cat, 2)]:
        tid = c.template_load(k, e, root)
        res = c.count(gid, tid, seed=23, n_iter=2, want_maps=True)
        assert res["maps"] == [O.count_maps(g, k, e, root, seed=23, j=j) for j in range(2)]
    c.close()


@pytest.mark.parametrize("fused", [0, 1])
def test_default_segments_with_hubs(fused):
    # default col_chunks: segmented task and unfused gathers, whole-row fused
    # kernels; rows of 8 colourings are large enough for several segments
    g = gg.rmat_graph(12, seed=47)
    k = 10
    broom = [(0, 1), (1, 2), (2, 3)] + [(0, j) for j in range(4, 10)]
    deg = np.diff(g.row_ptr)
    assert ((deg >= 64) & (deg <= 1024)).sum() > 20
    c = make_ctx(fused=fused, batch=8, block_vertices=1500)
    gid = c.graph_load(g)
    tid = c.template_load(k, broom, 0)
    res = c.count(gid, tid, seed=29, n_iter=8, want_maps=True)
    assert res["maps"] == [O.count_maps(g, k, broom, 0, seed=29, j=j) for j in range(8)]
    c.close()


@pytest.fixture(scope="module")
def hub_of_stars():
    # hub 0 - 300 middle vertices - 250 leaves each: aggregates ~75,300 at the hub
    M, P = 300, 250
    edges = [(0, 1 + i) for i in range(M)]
    nid = 1 + M
    for i in range(M):
        for _ in range(P):
            edges.append((1 + i, nid))
            nid += 1
    return gg.csr_from_edges(nid, np.array(edges))


@pytest.mark.parametrize("fused", [0, 1])
def test_mixed_width_steps(hub_of_stars, fused):
    # spider with five legs of length 2, rooted at its centre: the bounds after
    # 3, 4 and 5 legs are ~4e14, ~3e19 and ~2e24, so the root chain's steps run
    # at 1, 1, 1, 2 and 2 limbs with one-limb aggregates (the generic combine
    # multiplies 1x1 and 2x1 limbs into 2); the map counts exceed 2^64
    g = hub_of_stars
    spider = [(0, 1), (1, 2), (0, 3), (3, 4), (0, 5), (5, 6), (0, 7), (7, 8), (0, 9), (9, 10)]
    maps = [O.count_maps(g, 11, spider, 0, seed=3, j=j) for j in range(2)]
    assert max(maps) >= 1 << 64
    c = make_ctx(fused=fused, batch=2)
    gid = c.graph_load(g)
    tid = c.template_load(11, spider, 0)
    res = c.count(gid, tid, seed=3, n_iter=2, want_maps=True)
    assert res["limbs"] == 2 and res["maps"] == maps
    c.close()


@pytest.mark.parametrize("split", [8, 1 << 20])
def test_kernel_stats_time_heavy_vertices_apart(split):
    # the Algorithm 4 path (vertices with more than `split` neighbours) is its own
    # kind; with no such vertex it launches nothing
    g = gg.rmat_graph(10, seed=62)
    k, e = gg.template_edges("tree12")
    c = make_ctx(split_threshold=split, timing=1)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 1)
    c.count(gid, tid, seed=3, n_iter=2)
    st = c.kernel_stats()
    kinds = [n for n in st if n != "total_launches"]
    assert kinds == ["colour", "hist", "gather", "combine", "reduce", "fused", "select", "combine_hist", "heavy"]
    assert st["fused"]["launches"] > 0 and st["fused"]["bytes"] > 0
    if split == 8:
        assert st["heavy"]["launches"] > 0 and st["heavy"]["bytes"] > 0
    else:
        assert st["heavy"]["launches"] == 0
    assert sum(st[n]["launches"] for n in kinds) <= st["total_launches"]
    c.close()


@pytest.mark.parametrize("order", [0, 1])
def test_vertex_orders_give_identical_counts_and_samples(order):
    g = gg.rmat_graph(10, seed=61)
    k, e = gg.template_edges("caterpillar10")
    _, pv = O.count_maps(g, k, e, 2, seed=6, j=0, per_vertex=True)
    c = make_ctx(vertex_order=order, split_threshold=24)
    gid = c.graph_load(g)
    tid = c.template_load(k, e, 2)
    sample = list(range(0, g.n, 5))
    res = c.count(gid, tid, seed=6, n_iter=1, sample_vertices=sample, want_maps=True)
    assert res["maps"][0] == sum(pv)
    assert res["samples"][0] == [pv[v] for v in sample]
    c.close()


def test_limb_product_rate():
    # register-resident 64-bit multiply-adds: far above 1e11/s on any GB300
    c = make_ctx()
    r = c.limb_product_rate()
    assert 1e11 < r < 1e15
    c.close()
