"""Host-side checks that need no GPU: the C-ABI library loads and exports every
symbol of include/cc.h, the planner's cost model reproduces Table 4, the
library's automorphism count (AHU canonical forms) agrees with the oracle's
backtracking count, and the input generators behave."""
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import build as B
from paper_1804_09764_gb300 import cc
from paper_1804_09764_gb300 import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cc.load_library()


def header_functions():
    with open(os.path.join(ROOT, "include", "cc.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function(lib):
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(cc.EXPORTED) <= set(names)
    assert lib.cc_version().decode().startswith("cc-gb300")


def test_status_strings(lib):
    for code, name in cc.STATUS.items():
        assert lib.cc_status_string(code).decode() == name


def test_table4_cost_model():
    # Table 4 (Section 4.1): memory = sum C(k,|T_i|), computation = sum C(k,|T_i|) C(|T_i|,|T_i'|)
    rows = []
    with open(os.path.join(GOLDEN, "table4_cost.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    assert len(rows) == 3
    for name, k, mem, comp, edges in rows:
        e = [tuple(int(x) for x in p.split("-")) for p in edges.split(",")]
        assert cc.cc_template_cost(int(k), e, 0, 0) == (int(mem), int(comp)), name


def test_automorphisms_agree_with_oracle():
    for k in range(1, 13):
        for seed in range(5):
            e = gg.prufer_tree(k, 1000 + seed)
            assert cc.cc_template_automorphisms(k, e) == O.automorphisms(k, e)
    for name in ("P5", "caterpillar10", "tree12", "spider15"):
        k, e = gg.template_edges(name)
        assert cc.cc_template_automorphisms(k, e) == O.automorphisms(k, e)
    # stars: (k-1)! (not enumerated by the oracle)
    for k in (10, 14, 16):
        assert cc.cc_template_automorphisms(k, [(0, i) for i in range(1, k)]) == int(np.prod(range(1, k)))


def test_template_validation(lib):
    with pytest.raises(cc.CCError) as ei:
        cc.cc_template_cost(3, [(0, 1), (0, 1)], 0)
    assert ei.value.status == -3
    with pytest.raises(cc.CCError) as ei:
        cc.cc_template_cost(4, [(0, 1), (2, 3), (0, 1)], 0)
    assert ei.value.status == -3
    with pytest.raises(cc.CCError) as ei:
        cc.cc_template_cost(17, [(i, i + 1) for i in range(16)], 0)
    assert ei.value.status == -4


def test_generators_are_deterministic_and_simple():
    a = gg.rmat_graph(10, seed=3)
    b = gg.rmat_graph(10, seed=3)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    for g in (a, gg.er_graph(500, 8, seed=2), gg.cycle_graph(7), gg.complete_graph(6), gg.star_graph(9)):
        assert g.row_ptr[0] == 0 and g.row_ptr[-1] == g.col_idx.size
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        assert not np.any(src == g.col_idx)
        fwd = set(zip(src.tolist(), g.col_idx.tolist()))
        assert len(fwd) == g.col_idx.size
        assert all((v, u) in fwd for u, v in fwd)
    er = gg.er_graph(2000, 8, seed=1)
    assert er.m == 8000


def test_prufer_trees_are_trees():
    for k in range(2, 17):
        e = gg.prufer_tree(k, k)
        assert len(e) == k - 1
        assert O.automorphisms(k, e) >= 1  # raises if not a tree


# ------------------------------------------------ Algorithm 1's sample size

def _group_failure(s, k, eps):
    """Exact probability that the mean of s colourings misses (1 +- eps) N when
    G is T itself: one copy, colourful with probability p = k!/k^k, so the
    colourful count is Bernoulli(p) and the group mean is Binomial(s, p) / (s p)."""
    binom = pytest.importorskip("scipy.stats").binom
    p = math.factorial(k) / k ** k
    c = np.arange(s + 1)
    return float(binom.pmf(c, s, p)[np.abs(c / (s * p) - 1) > eps].sum())


@pytest.mark.parametrize("k,eps,delta", [(2, 0.5, 0.1), (3, 0.5, 0.05), (4, 1.0, 0.2), (5, 0.8, 0.1),
                                         (3, 0.25, 0.01), (6, 1.5, 0.3)])
def test_iterations_for_meets_the_guarantee_where_the_variance_bound_is_tight(lib, k, eps, delta):
    # G = T attains Var X / (E X)^2 = 1/p - 1, the bound the sample size rests on;
    # the failure probabilities there are computed exactly from binomial tails
    binom = pytest.importorskip("scipy.stats").binom
    n, t = cc.cc_iterations_for(k, eps, delta)
    s = n // t
    assert n == s * t and s >= 1 and t >= 1
    pg = _group_failure(s, k, eps)
    assert pg <= 0.25
    # the median of t group means is off only if at least half of the groups are
    assert binom.sf(math.ceil(t / 2) - 1, t, pg) <= delta


def test_iterations_for_pin_rejects_a_group_size_without_the_colourful_probability(lib):
    # a plausible slip, s = 4 / eps^2 (dropping 1/p - 1), fails the exact check
    k, eps = 5, 0.8
    assert _group_failure(math.ceil(4 / eps ** 2), k, eps) > 0.25


def test_iterations_for_limits_and_errors(lib):
    assert cc.cc_iterations_for(1, 0.1, 0.5)[0] == cc.cc_iterations_for(1, 0.1, 0.5)[1]  # k = 1: no variance
    n1, t1 = cc.cc_iterations_for(6, 0.5, 0.1)
    n2, t2 = cc.cc_iterations_for(6, 0.25, 0.1)
    n3, t3 = cc.cc_iterations_for(6, 0.5, 0.01)
    assert t1 == t2 and n2 > 3 * n1 and t3 > t1 and n3 > n1
    for k, eps, delta, status in [(0, 0.5, 0.1, -4), (17, 0.5, 0.1, -4), (4, 0.0, 0.1, -1), (4, -1.0, 0.1, -1),
                                  (4, 0.5, 0.0, -1), (4, 0.5, 1.0, -1), (4, float("nan"), 0.1, -1),
                                  (16, 1e-6, 1e-9, -11)]:
        with pytest.raises(cc.CCError) as ei:
            cc.cc_iterations_for(k, eps, delta)
        assert ei.value.status == status


def test_all_trees_counts_match_the_number_of_free_trees():
    # unlabelled trees on k vertices: 1, 1, 1, 2, 3, 6, 11 for k = 1..7 (Otter)
    for k, want in zip(range(1, 8), [1, 1, 1, 2, 3, 6, 11]):
        trees = gg.all_trees(k)
        assert len(trees) == want
        for e in trees:
            assert len(e) == k - 1
            assert O.automorphisms(k, e) >= 1  # a tree on 0..k-1 (the oracle checks connectivity)


def test_labelled_automorphisms_library_vs_oracle(lib):
    # AHU canonical forms with labels (library) against backtracking over
    # label-preserving bijections (oracle)
    import random

    rng = random.Random(5)
    for i in range(40):
        k = rng.randrange(2, 11)
        e = gg.prufer_tree(k, 700 + i)
        lab = [rng.randrange(3) for _ in range(k)]
        assert cc.cc_template_automorphisms_labelled(k, e, lab) == O.automorphisms(k, e, lab)
    for name in ["caterpillar10", "tree12", "spider15"]:
        k, e = gg.template_edges(name)
        assert cc.cc_template_automorphisms_labelled(k, e, [0] * k) == cc.cc_template_automorphisms(k, e)


def test_header_is_plain_c_and_cpp(tmp_path):
    # include/cc.h is the C ABI: it must compile as strict C11 and as C++
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    src = tmp_path / "t.c"
    src.write_text('#include "cc.h"\nint main(void) { cc_options o; cc_default_options(&o); '
                   'return (int)sizeof(cc_plan_info) > 0 ? 0 : 1; }\n')
    inc = os.path.join(ROOT, "include")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                           "-I", inc, str(src)])
    if shutil.which("g++"):
        subprocess.check_call(["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-x", "c++", "-I", inc,
                               str(src)])


def test_c_caller_compiles_and_links_against_the_library(lib, tmp_path):
    # the boundary is a C ABI: a plain C program builds against include/cc.h
    # and the shared library (running it needs a GPU)
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    build_dir = os.path.dirname(cc.LIB_PATH)
    exe = tmp_path / "c_abi_example"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi_example.c"), "-L", build_dir, "-lcc_gb300",
                           f"-Wl,-rpath,{build_dir}", "-o", str(exe)])
    assert exe.exists()


def _isomorphic_brute(k, e1, e2, l1=None, l2=None):
    """Is there a vertex bijection (label-preserving when labels are given)
    mapping the edges of e1 onto those of e2?  Plain search over k! maps."""
    import itertools

    s2 = {frozenset(x) for x in e2}
    for perm in itertools.permutations(range(k)):
        if l1 is not None and any(l1[v] != l2[perm[v]] for v in range(k)):
            continue
        if all(frozenset((perm[a], perm[b])) in s2 for a, b in e1):
            return True
    return False


def test_canonical_form_is_the_isomorphism_class(lib):
    # the key by which served requests of isomorphic templates share passes
    import itertools
    import random

    # over all Pruefer sequences on k vertices the forms take as many values
    # as there are unlabelled trees (Otter: 1, 2, 3, 6, 11 for k = 3..7)
    for k, want in zip(range(3, 8), [1, 2, 3, 6, 11]):
        forms = {cc.cc_template_canonical_form(k, gg._prufer_decode(k, seq))
                 for seq in itertools.product(range(k), repeat=k - 2)}
        assert len(forms) == want
    rng = random.Random(17)
    for i in range(40):
        k = rng.randrange(4, 8)
        e1, e2 = gg.prufer_tree(k, 900 + i), gg.prufer_tree(k, 950 + i)
        perm = list(range(k))
        rng.shuffle(perm)
        e1p = [(perm[a], perm[b]) for a, b in e1]
        assert cc.cc_template_canonical_form(k, e1p) == cc.cc_template_canonical_form(k, e1)
        same = cc.cc_template_canonical_form(k, e1) == cc.cc_template_canonical_form(k, e2)
        assert same == _isomorphic_brute(k, e1, e2)
        # labelled: the forms agree exactly when a label-preserving map exists
        l1 = [rng.randrange(2) for _ in range(k)]
        l2 = [rng.randrange(2) for _ in range(k)]
        same = cc.cc_template_canonical_form(k, e1, l1) == cc.cc_template_canonical_form(k, e1p, l2)
        l1p = [0] * k
        for v in range(k):
            l1p[perm[v]] = l1[v]
        assert same == _isomorphic_brute(k, e1, e1p, l1, l2)
        assert cc.cc_template_canonical_form(k, e1p, l1p) == cc.cc_template_canonical_form(k, e1, l1)
