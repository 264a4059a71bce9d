"""The kernels of the R-MAT scale-22 / tree-12 benchmark, against the oracle.

At scale 22 the homomorphism bounds give the tree-12 plan (root 1) these
integer widths: the 66-, 792- and 924-column tables one 64-bit limb, the
495-column table two, the root chain's gather step two and its total three.
So the benchmark's fused kind runs the chain kernel at <Ls, Lf, Ld> = <2,2,3>
(root chain), <1,2,2> (the 495-column chain) and <1,1,1> (the 792-column
chain), and the plain fused gather + select at <1,1> (the 924-column chain),
with heavy vertices (more than 4096 neighbours) on the task path.

R-MAT scale 22 is far too large for the oracle, so these tests use a graph
whose bounds give the same widths: K_{500,6000} beside R-MAT scale 11
(tests/golden/make_tree12_widths.py explains the choice).  Its oracle counts
take about two minutes per colouring, so they are stored in
tests/golden/tree12_widths.json, written by that script from the oracle
alone.  The tests check that the plan and the launched instantiations are the
benchmark's, then compare maps, copies and sampled per-vertex counts with the
oracle's element by element (Eq. 1 and Eq. 3, Section 2.1)."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1804_09764_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "tree12_widths.json")

# (template vertex of the chain, step) -> (path, kernel limb arguments)
EXPECTED_PATHS = {
    (5, 0): ("leaf_select", (0, 0, 1)),
    (4, 0): ("chain_kernel", (1, 1, 1)),
    (3, 0): ("fused_select", (1, 0, 1)),
    (2, 0): ("chain_kernel", (1, 2, 2)),
    (1, 0): ("chain_kernel", (2, 2, 3)),
}
# the chains' table widths: 66, 792, 924 and 495 columns, then the root's total
EXPECTED_CHAIN_LIMBS = {5: 1, 4: 1, 3: 1, 2: 2, 1: 3}
EXPECTED_FUSED = {"gather_select_chain_kernel<2,2,3>", "gather_select_chain_kernel<1,2,2>",
                  "gather_select_chain_kernel<1,1,1>", "gather_select_kernel<1,1>"}


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def graph(gold):
    g = gg.disjoint_union(gg.complete_bipartite_graph(500, 6000), gg.rmat_graph(11, seed=11))
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(g.col_idx, dtype=np.int32).tobytes())
    assert h.hexdigest() == gold["graph"]["sha256"], "generator output differs from the stored graph"
    return g


def run(graph, gold, **kw):
    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    k, e = gg.template_edges("tree12")
    c = cc.Context(budget_bytes=8 << 30, timing=1, **kw)
    gid = c.graph_load(graph)
    tid = c.template_load(k, e, gold["root"])
    res = c.count(gid, tid, seed=gold["seed"], n_iter=len(gold["colourings"]), first_iter=gold["colourings"][0],
                  want_maps=True, sample_vertices=gold["sample_vertices"])
    steps = c.plan_steps(gid, tid)
    inst = c.kernel_instances()
    info = c.plan_info(gid, tid)
    c.close()
    return res, steps, inst, info


def check_against_oracle(res, gold):
    maps = [int(m, 16) for m in gold["maps"]]
    aut = gold["aut"]
    assert res["maps"] == maps
    assert res["exact"] == 1 and res["counts"] == [m // aut for m in maps]
    for j, row in enumerate(gold["sample_maps"]):
        assert res["samples"][j] == [int(x, 16) for x in row], f"colouring {j}"


def test_benchmark_widths_and_kernels_match_oracle(graph, gold):
    # the benchmark's configuration: defaults (split 4096, column segments
    # auto, degree ordering, fused kernels), one colouring per pass, the
    # vertices streamed in four blocks with a ragged tail
    res, steps, inst, info = run(graph, gold, batch=1, block_vertices=2100)
    assert info["limbs_root"] == 3 and info["split_threshold"] == 4096
    assert info["n_blocks"] == 4 and info["batch"] == 1
    by = {(s["vertex"], s["step"]): s for s in steps}
    for key, (path, limbs) in EXPECTED_PATHS.items():
        assert (by[key]["path"], by[key]["kernel_limbs"]) == (path, limbs), key
    for s in steps:
        assert s["chain_limbs"] == EXPECTED_CHAIN_LIMBS[s["vertex"]], s
    # the root chain's leaf steps run inside its chain kernel
    assert [s["path"] for s in steps if s["vertex"] == 1] == ["chain_kernel"] + ["in_chain"] * 3
    assert set(inst["fused"]) == EXPECTED_FUSED
    # the 500 vertices of degree 6000 take the task path (Algorithm 4)
    assert "gather_tasks_kernel<2,3>" in inst["heavy"] and "combine_hist_kernel<3,3>" in inst["heavy"]
    check_against_oracle(res, gold)


def test_benchmark_kernels_with_batched_colourings(graph, gold):
    # both colourings in one pass (rows of two colourings) and one block
    res, steps, inst, info = run(graph, gold)
    assert info["batch"] == 2 and info["n_blocks"] == 1
    assert set(inst["fused"]) == EXPECTED_FUSED
    check_against_oracle(res, gold)
