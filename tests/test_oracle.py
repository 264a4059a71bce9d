"""Pins for the CPU oracle: it is checked here against things other than itself.

* brute-force enumeration of colourful labelled maps on tiny graphs, every root
  (Section 2: non-induced embeddings; Section 2.1: colourful, rooted counts),
* the exact identity obtained by summing over all k^n colourings
  (Section 2.1: an embedding is colourful with probability k!/k^k),
* closed forms (paths on cycles, any tree on K_n, stars on stars),
* the published first output of SplitMix64 (colouring rule),
* 256-bit arithmetic against Python integers,
* |Aut(T)| against permutation brute force.
"""
import itertools
import math
import os
import random
from collections import Counter

import numpy as np
import pytest

import oracle as O
from paper_1804_09764_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SMALL_TEMPLATES = {
    "P2": (2, [(0, 1)]),
    "P3": (3, [(0, 1), (1, 2)]),
    "P4": (4, [(0, 1), (1, 2), (2, 3)]),
    "star4": (4, [(0, 1), (0, 2), (0, 3)]),
    "spider5": (5, [(0, 1), (1, 2), (0, 3), (0, 4)]),
    "cat6": (6, [(0, 1), (1, 2), (2, 3), (1, 4), (2, 5)]),
}


def brute_maps(graph, colours, k, edges):
    """Injective maps f: V_T -> V with every template edge on a graph edge and
    k distinct colours (Section 2 definition, enumerated)."""
    nb = [set(graph.neighbours(v).tolist()) for v in range(graph.n)]
    cnt = 0
    for img in itertools.permutations(range(graph.n), k):
        if len({colours[v] for v in img}) != k:
            continue
        if all(img[b] in nb[img[a]] for a, b in edges):
            cnt += 1
    return cnt


def brute_copies_uncoloured(graph, k, edges):
    nb = [set(graph.neighbours(v).tolist()) for v in range(graph.n)]
    maps = sum(1 for img in itertools.permutations(range(graph.n), k)
               if all(img[b] in nb[img[a]] for a, b in edges))
    return maps // brute_aut(k, edges)


def brute_aut(k, edges):
    E = {frozenset(e) for e in edges}
    return sum(1 for p in itertools.permutations(range(k))
               if all(frozenset((p[a], p[b])) in E for a, b in edges))


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- colouring

def test_splitmix64_published_first_output():
    rows = dict(read_golden("splitmix64.txt"))
    assert O.splitmix64(int(rows["state"], 0)) == int(rows["first_output"], 0)


def test_colour_rule_composition_and_range():
    # h = F(F(F(seed) + j) + id); col = floor(h k / 2^64)
    M = 2 ** 64
    for seed, j, v, k in [(0, 0, 0, 5), (7, 3, 123456, 12), (2 ** 64 - 1, 9, 2 ** 40, 15)]:
        h = O.splitmix64((O.splitmix64((O.splitmix64(seed) + j) % M) + v) % M)
        assert O.colour(seed, j, [v], k)[0] == (h * k) >> 64


@pytest.mark.parametrize("k", [2, 5, 12, 16])
def test_colour_rule_is_uniform(k):
    n = 60000
    col = O.colour(11, 4, np.arange(n), k)
    assert col.max() < k
    obs = np.bincount(col, minlength=k)
    exp = n / k
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    # chi-square with k-1 dof; 99.9% quantile is below 3*k + 25 for k <= 16
    assert chi2 < 3 * k + 25


# ----------------------------------------------------------------- integers

def test_u256_arithmetic_matches_python_integers():
    rng = random.Random(5)
    M = 1 << 256
    for _ in range(300):
        bits_a = rng.choice([1, 63, 64, 65, 127, 128, 129, 191, 200, 255, 256])
        bits_b = rng.choice([1, 64, 100, 128, 192, 256])
        a = rng.getrandbits(bits_a)
        b = rng.getrandbits(bits_b)
        assert O.u256_mul(a, b) == (a * b) % M
        assert O.u256_add(a, b) == (a + b) % M


# ----------------------------------------------------------------- automorphisms

def test_automorphisms_against_permutations():
    for k in range(1, 9):
        for seed in range(6):
            e = gg.prufer_tree(k, seed)
            assert O.automorphisms(k, e) == brute_aut(k, e)


def test_automorphisms_of_workload_templates():
    # P5: reflection (2).  caterpillar10: 3 leaves on each of vertices 1 and 3,
    # swapped by the reflection: 3!*3!*2 = 72.  tree12: 3 leaves on 1 (3!) and 2
    # on 4 (2!) = 12.  spider15: three legs of length 3 (3!) and two of length
    # 2 (2!) = 12.
    expect = {"P5": 2, "caterpillar10": 72, "tree12": 12, "spider15": 12}
    for name, a in expect.items():
        assert O.automorphisms(*gg.template_edges(name)) == a


# ----------------------------------------------------------------- brute force

@pytest.mark.parametrize("name", list(SMALL_TEMPLATES))
def test_dp_matches_brute_force_every_root(name):
    k, edges = SMALL_TEMPLATES[name]
    rng = np.random.default_rng(hash(name) % 1000)
    for trial in range(3):
        g = gg.random_graph_gnp(8, 0.5, seed=trial * 31 + k)
        colours = rng.integers(0, k, g.n).astype(np.uint8)
        bf = brute_maps(g, colours, k, edges)
        aut = O.automorphisms(k, edges)
        assert bf % aut == 0
        for root in range(k):
            assert O.count_maps(g, k, edges, root, colours=colours) == bf


def test_dp_matches_brute_force_random_trees_seeded_colouring():
    for seed in range(8):
        k = 3 + seed % 4
        edges = gg.prufer_tree(k, seed + 100)
        g = gg.random_graph_gnp(8, 0.55, seed=seed)
        colours = O.colour(seed, 2, np.arange(g.n), k)
        bf = brute_maps(g, colours, k, edges)
        for root in range(k):
            assert O.count_maps(g, k, edges, root, seed=seed, j=2) == bf


def test_per_vertex_counts_match_brute_force_rooted():
    k, edges = SMALL_TEMPLATES["spider5"]
    g = gg.random_graph_gnp(8, 0.6, seed=3)
    colours = np.array([0, 1, 2, 3, 4, 0, 1, 2], dtype=np.uint8)
    nb = [set(g.neighbours(v).tolist()) for v in range(g.n)]
    for root in range(k):
        _, pv = O.count_maps(g, k, edges, root, colours=colours, per_vertex=True)
        for v in range(g.n):
            cnt = 0
            for img in itertools.permutations(range(g.n), k):
                if img[root] != v or len({colours[x] for x in img}) != k:
                    continue
                if all(img[b] in nb[img[a]] for a, b in edges):
                    cnt += 1
            assert pv[v] == cnt


# ----------------------------------------------------------------- invariants

def test_sum_over_all_colourings_recovers_exact_count():
    # sum over the k^n colourings of colourful copies = #copies * k! * k^(n-k)
    n, k = 6, 4
    edges = [(0, 1), (1, 2), (1, 3)]
    g = gg.random_graph_gnp(n, 0.6, seed=9)
    aut = O.automorphisms(k, edges)
    total = 0
    for col in itertools.product(range(k), repeat=n):
        total += O.count_maps(g, k, edges, 1, colours=np.array(col, dtype=np.uint8)) // aut
    assert total == brute_copies_uncoloured(g, k, edges) * math.factorial(k) * k ** (n - k)


def test_sum_over_all_colourings_on_complete_graph_closed_form():
    # K_n has n!/(n-k)!/|Aut| copies of any k-vertex tree
    n, k = 6, 4
    edges = [(0, 1), (1, 2), (2, 3)]
    g = gg.complete_graph(n)
    aut = O.automorphisms(k, edges)
    total = sum(O.count_maps(g, k, edges, 0, colours=np.array(col, dtype=np.uint8)) // aut
                for col in itertools.product(range(k), repeat=n))
    copies = math.factorial(n) // math.factorial(n - k) // aut
    assert total == copies * math.factorial(k) * k ** (n - k)


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n,k", [(11, 2), (11, 4), (13, 5), (9, 8)])
def test_path_on_cycle_counts_colourful_windows(n, k):
    edges = [(i, i + 1) for i in range(k - 1)]
    g = gg.cycle_graph(n)
    colours = O.colour(3, n, np.arange(n), k)
    windows = sum(1 for i in range(n) if len({colours[(i + t) % n] for t in range(k)}) == k)
    maps = O.count_maps(g, k, edges, 0, colours=colours)
    assert maps // O.automorphisms(k, edges) == windows


@pytest.mark.parametrize("name", ["P4", "star4", "spider5", "cat6"])
def test_any_tree_on_complete_graph(name):
    # colourful copies on K_n = (k!/|Aut|) * prod_c n_c (one vertex per colour class)
    k, edges = SMALL_TEMPLATES[name]
    n = 13
    g = gg.complete_graph(n)
    colours = O.colour(17, k, np.arange(n), k)
    cnt = Counter(colours.tolist())
    aut = O.automorphisms(k, edges)
    expect = math.factorial(k) // aut * math.prod(cnt[c] for c in range(k))
    assert O.count_maps(g, k, edges, 0, colours=colours) == expect * aut


@pytest.mark.parametrize("k,leaves", [(10, 3000), (14, 4000)])
def test_star_on_star_graph_wide_counts(k, leaves):
    # star template (centre 0) on K_{1,N}: colourful copies = prod over colours c
    # other than the hub's of the number of leaves coloured c.  These counts pass
    # 2^64 (k=10) and 2^128 (k=14), exercising the wide arithmetic.
    edges = [(0, i) for i in range(1, k)]
    g = gg.star_graph(leaves)
    colours = O.colour(5, 0, np.arange(g.n), k)
    cnt = Counter(colours[1:].tolist())
    expect = math.prod(cnt[c] for c in range(k) if c != colours[0])
    aut = math.factorial(k - 1)        # the k-1 leaves permute freely
    if k <= 10:                        # the backtracking count enumerates every automorphism
        assert O.automorphisms(k, edges) == aut
    maps = O.count_maps(g, k, edges, 0, colours=colours)
    assert maps == expect * aut
    assert maps.bit_length() > (64 if k == 10 else 128)


def test_single_vertex_and_single_edge():
    g = gg.er_graph(50, 4, seed=2)
    assert O.count_maps(g, 1, [], 0, seed=1) == g.n
    col = O.colour(1, 0, np.arange(g.n), 2)
    colourful_edges = sum(1 for v in range(g.n) for u in g.neighbours(v) if u > v and col[u] != col[v])
    for root in (0, 1):
        assert O.count_maps(g, 2, [(0, 1)], root, seed=1, j=0) == 2 * colourful_edges


def test_partition_invariance_on_rmat():
    g = gg.rmat_graph(8, seed=4)
    k, edges = gg.template_edges("caterpillar10")
    vals = {O.count_maps(g, k, edges, r, seed=3, j=1) for r in range(k)}
    assert len(vals) == 1


def test_subgraph_ids_keep_original_colours():
    # running on an induced subgraph with the original ids reproduces the colours
    g = gg.er_graph(40, 3, seed=1)
    ids = np.arange(g.n, dtype=np.int64)
    k, edges = SMALL_TEMPLATES["P4"]
    assert O.count_maps(g, k, edges, 0, seed=8, j=5, ids=ids) == O.count_maps(g, k, edges, 0, seed=8, j=5)


# ----------------------------------------------------------------- estimate

def test_estimate_and_median_of_means():
    assert O.estimate(6, 3) == pytest.approx(6 * 27 / 6)
    assert O.median_of_means([1.0, 2.0, 3.0, 10.0], 1) == pytest.approx(4.0)
    assert O.median_of_means([1.0, 3.0, 5.0, 7.0, 100.0, 200.0], 3) == pytest.approx(6.0)
    assert O.median_of_means([1.0, 2.0, 3.0, 4.0], 4) == pytest.approx(2.5)


def test_unbiasedness_over_all_colourings_small():
    # mean over all colourings of est_j equals the exact number of copies
    n, k = 5, 3
    edges = [(0, 1), (1, 2)]
    g = gg.random_graph_gnp(n, 0.7, seed=1)
    aut = O.automorphisms(k, edges)
    ests = [O.estimate(O.count_maps(g, k, edges, 1, colours=np.array(c, dtype=np.uint8)) // aut, k)
            for c in itertools.product(range(k), repeat=n)]
    assert math.fsum(ests) / len(ests) == pytest.approx(brute_copies_uncoloured(g, k, edges), rel=1e-12)


# ----------------------------------------------------------------- labelled templates
# Vertex labels on G and T: a counted map sends every template vertex to a
# graph vertex with the same label (the labelled templates of SAHAD, cited in
# the related work); copies divide by the label-preserving automorphisms.

def brute_maps_labelled(graph, colours, k, edges, glab, tlab):
    nb = [set(graph.neighbours(v).tolist()) for v in range(graph.n)]
    cnt = 0
    for img in itertools.permutations(range(graph.n), k):
        if any(glab[img[x]] != tlab[x] for x in range(k)):
            continue
        if len({colours[v] for v in img}) != k:
            continue
        if all(img[b] in nb[img[a]] for a, b in edges):
            cnt += 1
    return cnt


def brute_aut_labelled(k, edges, lab):
    E = {frozenset(e) for e in edges}
    return sum(1 for p in itertools.permutations(range(k))
               if all(lab[p[x]] == lab[x] for x in range(k))
               and all(frozenset((p[a], p[b])) in E for a, b in edges))


@pytest.mark.parametrize("name", ["P3", "P4", "star4", "spider5"])
def test_labelled_dp_matches_brute_force_every_root(name):
    k, edges = SMALL_TEMPLATES[name]
    rng = random.Random(sum(map(ord, name)) * 7919)
    g = gg.random_graph_gnp(9, 0.5, seed=31)
    for trial in range(3):
        colours = [rng.randrange(k) for _ in range(g.n)]
        glab = [rng.randrange(2) for _ in range(g.n)]
        tlab = [rng.randrange(2) for _ in range(k)]
        bf = brute_maps_labelled(g, colours, k, edges, glab, tlab)
        for root in range(k):
            assert O.count_maps(g, k, edges, root, colours=colours, glabels=glab, tlabels=tlab) == bf


def test_labelled_counts_over_all_template_labellings_sum_to_unlabelled():
    # every map induces exactly one labelling of T (the labels of its image),
    # so summing over all labellings of the template gives the unlabelled count
    k, edges = SMALL_TEMPLATES["cat6"]
    g = gg.rmat_graph(7, seed=5)
    glab = np.random.default_rng(3).integers(0, 2, g.n)
    total = sum(O.count_maps(g, k, edges, 1, seed=7, j=0, glabels=glab, tlabels=list(t))
                for t in itertools.product(range(2), repeat=k))
    assert total == O.count_maps(g, k, edges, 1, seed=7, j=0)


def test_labelled_automorphisms_against_permutations():
    rng = random.Random(11)
    for name, (k, e) in SMALL_TEMPLATES.items():
        for _ in range(4):
            lab = [rng.randrange(2) for _ in range(k)]
            assert O.automorphisms(k, e, lab) == brute_aut_labelled(k, e, lab)
        assert O.automorphisms(k, e, [0] * k) == O.automorphisms(k, e)


# ----------------------------------------------------------------- the table gather on its own

def _ints(X):
    return [[sum(int(X[u, c, i]) << (64 * i) for i in range(X.shape[2])) for c in range(X.shape[1])]
            for u in range(X.shape[0])]


def test_neighbour_sum_closed_forms_on_a_star():
    # hub 0 and leaves 1..N: the hub sums the leaves' rows, every leaf gets the hub's row
    N, L = 6, 2
    g = gg.star_graph(N)
    X = np.random.default_rng(1).integers(0, 2 ** 63, size=(N + 1, 3, L), dtype=np.uint64)
    out = _ints(O.neighbour_sum(g, X, L))
    x = _ints(X)
    M = 1 << (64 * L)
    assert out[0] == [sum(x[u][c] for u in range(1, N + 1)) % M for c in range(3)]
    for leaf in range(1, N + 1):
        assert out[leaf] == x[0]


def test_neighbour_sum_wraps_modulo_its_width():
    g = gg.star_graph(2)
    for L in (1, 2, 3):
        X = np.full((3, 1, L), np.uint64(2 ** 64 - 1))
        assert _ints(O.neighbour_sum(g, X, L))[0][0] == (1 << (64 * L)) - 2


def test_neighbour_sum_of_colour_indicators_gives_edge_map_counts():
    # gathering the one-hot colour table gives each vertex its neighbours'
    # colour histogram; the colours other than its own count the colourful
    # maps of an edge rooted at it (the C dynamic program, per vertex)
    g = gg.rmat_graph(8, seed=12)
    k = 2  # the edge template's colours
    colours = O.colour(9, 0, range(g.n), k)
    X = np.zeros((g.n, k, 1), dtype=np.uint64)
    X[np.arange(g.n), colours.astype(np.int64), 0] = 1
    hist = O.neighbour_sum(g, X, 1)[:, :, 0]
    assert (hist.sum(axis=1) == np.diff(g.row_ptr)).all()
    _, pv = O.count_maps(g, 2, [(0, 1)], 0, colours=colours, per_vertex=True)
    assert pv == [int(hist[v].sum() - hist[v, colours[v]]) for v in range(g.n)]


def test_run_reports_brute_force_copies_per_colouring():
    # Algorithm 1 over colourings: per colouring, copies = colourful maps / |Aut|
    k, edges = SMALL_TEMPLATES["star4"]
    g = gg.random_graph_gnp(8, 0.6, seed=41)
    out = O.run(g, k, edges, seed=3, n_iter=4, root=0, first_iter=2)
    aut = brute_aut(k, edges)
    assert out["aut"] == aut
    for j in range(4):
        colours = O.colour(3, 2 + j, range(g.n), k)
        assert out["copies"][j] == brute_maps(g, colours, k, edges) // aut
    assert out["mean"] == pytest.approx(sum(c * k ** k / math.factorial(k) for c in out["copies"]) / 4, rel=1e-12)
    with pytest.raises(ArithmeticError):
        O.copies_from_maps(7, 2)
