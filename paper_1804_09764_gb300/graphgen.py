"""Seeded synthetic inputs: graphs in CSR form and tree templates.

This module is shared by the CPU oracle and by the CUDA path.  It holds no
arithmetic of the colour-coding method itself: it only builds graphs and
templates.  The paper's datasets (Section 4.1, Table 3) are not available, so
seeded R-MAT graphs (Chakrabarti et al., the generator the paper uses for its
RMAT-250M/500M inputs) and Erdos-Renyi graphs stand in for them.

Conventions (Section 2: undirected graph, N(v) excludes v):
  * CSR with int64 ``row_ptr`` (n+1) and int32 ``col_idx`` (2m); both
    directions of every undirected edge are present; no self-loops, no
    duplicate edges; each neighbour list is sorted ascending.
  * Isolated vertices stay in the vertex set.

R-MAT recipe: exactly ``edge_factor * 2**scale`` edge samples, each drawn bit
by bit with quadrant probabilities (a, b, c, d); self-loops and duplicates are
dropped (so m is below the nominal count) and vertex labels are then permuted
by a seeded random permutation (Graph500 practice) so that hubs are not
clustered at low labels.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSRGraph", "csr_from_edges", "er_graph", "rmat_graph", "cycle_graph",
    "complete_graph", "star_graph", "prufer_tree", "TEMPLATES", "template_edges",
    "random_graph_gnp", "complete_bipartite_graph", "disjoint_union",
]


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent difference)."""
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


class CSRGraph:
    """Undirected graph in symmetric CSR form."""

    def __init__(self, n: int, row_ptr: np.ndarray, col_idx: np.ndarray, name: str = ""):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.name = name

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return int(self.row_ptr[-1]) // 2

    @property
    def nnz(self) -> int:
        """Number of directed edges (2m)."""
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def neighbours(self, v: int) -> np.ndarray:
        return self.col_idx[self.row_ptr[v]:self.row_ptr[v + 1]]

    def __repr__(self) -> str:
        return f"CSRGraph({self.name!r}, n={self.n}, m={self.m})"


def _csr_from_unique_pairs(n: int, lo: np.ndarray, hi: np.ndarray, name: str) -> CSRGraph:
    """lo < hi, unique pairs -> symmetric CSR with sorted neighbour lists."""
    lo = lo.astype(np.int64, copy=False)
    hi = hi.astype(np.int64, copy=False)
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    key = src * n + dst
    key.sort()
    src = key // n
    dst = (key - src * n).astype(np.int32)
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSRGraph(n, row_ptr, dst, name)


def csr_from_edges(n: int, edges, name: str = "") -> CSRGraph:
    """Build a CSR graph from an iterable/array of undirected edges.

    Self-loops are dropped and duplicate edges merged.
    """
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if e.size and (e.min() < 0 or e.max() >= n):
        raise ValueError("edge endpoint out of range")
    e = e[e[:, 0] != e[:, 1]]
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    key = _sorted_unique(lo * n + hi)
    return _csr_from_unique_pairs(n, key // n, key % n, name)


def er_graph(n: int, avg_degree: float, seed: int) -> CSRGraph:
    """Erdos-Renyi G(n, m): the first m = n*avg_degree/2 distinct non-loop
    pairs in draw order of a seeded uniform pair stream."""
    m = int(round(n * avg_degree / 2))
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")
    rng = np.random.default_rng(seed)
    drawn = np.empty(0, dtype=np.int64)
    while True:
        cnt = int(1.25 * m) + 64
        a = rng.integers(0, n, size=cnt)
        b = rng.integers(0, n, size=cnt)
        ok = a != b
        a, b = a[ok], b[ok]
        drawn = np.concatenate([drawn, np.minimum(a, b) * n + np.maximum(a, b)])
        order = np.argsort(drawn, kind="stable")
        srt = drawn[order]
        first = np.ones(srt.size, dtype=bool)
        first[1:] = srt[1:] != srt[:-1]
        first_pos = np.sort(order[first])          # draw positions of first occurrences
        if first_pos.size >= m:
            keys = np.sort(drawn[first_pos[:m]])
            break
    return _csr_from_unique_pairs(n, keys // n, keys % n, f"er_n{n}_d{avg_degree}_s{seed}")


def random_graph_gnp(n: int, p: float, seed: int) -> CSRGraph:
    """G(n, p) on tiny n (used for brute-force tests)."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(iu[0].size) < p
    return _csr_from_unique_pairs(n, iu[0][keep], iu[1][keep], f"gnp_n{n}_p{p}_s{seed}")


def rmat_graph(scale: int, seed: int, edge_factor: int = 16,
               a: float = 0.57, b: float = 0.19, c: float = 0.19,
               permute: bool = True, chunk: int = 1 << 24) -> CSRGraph:
    """Seeded R-MAT graph on 2**scale vertices (d = 1 - a - b - c).

    Each of the edge_factor * 2**scale samples picks, level by level, one of the
    four quadrants with probabilities (a, b, c, d) from a uniform 32-bit draw.
    """
    if scale > 31:
        raise ValueError("scale must be <= 31")
    n = 1 << scale
    total = edge_factor << scale
    rng = np.random.default_rng(seed)
    two32 = float(1 << 32)
    t_a = np.uint32(min(int(a * two32), (1 << 32) - 1))
    t_ab = np.uint32(min(int((a + b) * two32), (1 << 32) - 1))
    t_abc = np.uint32(min(int((a + b + c) * two32), (1 << 32) - 1))
    keys = []
    done = 0
    while done < total:
        cnt = min(chunk, total - done)
        src = np.zeros(cnt, dtype=np.uint32)
        dst = np.zeros(cnt, dtype=np.uint32)
        for bit in range(scale):
            r = rng.integers(0, 1 << 32, size=cnt, dtype=np.uint32)
            down = r >= t_ab                          # quadrants c, d
            right = (r >= t_a) & (r < t_ab)           # quadrant b
            right |= r >= t_abc                       # quadrant d
            src |= down.astype(np.uint32) << np.uint32(bit)
            dst |= right.astype(np.uint32) << np.uint32(bit)
        keep = src != dst
        lo = np.minimum(src[keep], dst[keep]).astype(np.int64)
        hi = np.maximum(src[keep], dst[keep]).astype(np.int64)
        keys.append(_sorted_unique(lo * n + hi))
        done += cnt
    key = _sorted_unique(np.concatenate(keys)) if len(keys) > 1 else keys[0]
    lo = key >> scale
    hi = key & (n - 1)
    if permute:
        perm = np.random.default_rng(seed ^ 0x5EED5EED).permutation(n).astype(np.int64)
        lo, hi = perm[lo], perm[hi]
        l2 = np.minimum(lo, hi)
        h2 = np.maximum(lo, hi)
        lo, hi = l2, h2
    return _csr_from_unique_pairs(n, lo, hi, f"rmat_s{scale}_s{seed}")


def cycle_graph(n: int) -> CSRGraph:
    v = np.arange(n)
    return csr_from_edges(n, np.stack([v, (v + 1) % n], 1), f"cycle{n}")


def complete_graph(n: int) -> CSRGraph:
    iu = np.triu_indices(n, 1)
    return _csr_from_unique_pairs(n, iu[0], iu[1], f"K{n}")


def star_graph(leaves: int) -> CSRGraph:
    """K_{1,leaves}: hub 0 joined to vertices 1..leaves."""
    v = np.arange(1, leaves + 1)
    return csr_from_edges(leaves + 1, np.stack([np.zeros_like(v), v], 1), f"star{leaves}")


def complete_bipartite_graph(c: int, N: int) -> CSRGraph:
    """K_{c,N}: vertices 0..c-1 (degree N) each joined to all of c..c+N-1 (degree c)."""
    lo = np.repeat(np.arange(c, dtype=np.int64), N)
    hi = np.tile(np.arange(c, c + N, dtype=np.int64), c)
    return _csr_from_unique_pairs(c + N, lo, hi, f"K{c},{N}")


def disjoint_union(*graphs: CSRGraph) -> CSRGraph:
    """The graphs side by side: the vertices of graphs[i] follow those of
    graphs[i-1], and no edge joins two of them."""
    n = sum(g.n for g in graphs)
    rp = [np.zeros(1, dtype=np.int64)]
    ci = []
    vo = eo = 0
    for g in graphs:
        rp.append(g.row_ptr[1:] + eo)
        ci.append(g.col_idx.astype(np.int64) + vo)
        vo += g.n
        eo += g.nnz
    col = np.concatenate(ci).astype(np.int32) if ci else np.zeros(0, dtype=np.int32)
    return CSRGraph(n, np.concatenate(rp), col, "+".join(g.name for g in graphs))


def prufer_tree(k: int, seed: int) -> list[tuple[int, int]]:
    """Uniform labelled tree on k vertices from a seeded Pruefer sequence.

    Decoded with the standard smallest-leaf rule.
    """
    if k == 1:
        return []
    if k == 2:
        return [(0, 1)]
    rng = np.random.default_rng(seed)
    return _prufer_decode(k, [int(x) for x in rng.integers(0, k, size=k - 2)])


def _tree_form(k: int, edges) -> str:
    """Canonical string of an unlabelled tree: nested sorted child forms from
    its centre (the smaller of the two forms for a bicentral tree)."""
    adj = [[] for _ in range(k)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    deg = [len(x) for x in adj]
    layer = [v for v in range(k) if deg[v] <= 1]
    left = k
    while left > 2:
        left -= len(layer)
        nxt = []
        for v in layer:
            for u in adj[v]:
                deg[u] -= 1
                if deg[u] == 1:
                    nxt.append(u)
        layer = nxt

    def form(v, parent):
        return "(" + "".join(sorted(form(u, v) for u in adj[v] if u != parent)) + ")"

    return min(form(c, -1) for c in layer)


def all_trees(k: int) -> list[list[tuple[int, int]]]:
    """One labelled representative of every tree on k vertices (k <= 8), in
    the order of their first Pruefer sequence (lexicographic)."""
    import itertools

    if not 1 <= k <= 8:
        raise ValueError("all_trees enumerates Pruefer sequences: k must be in 1..8")
    if k <= 2:
        return [[] if k == 1 else [(0, 1)]]
    seen, out = set(), []
    for seq in itertools.product(range(k), repeat=k - 2):
        e = _prufer_decode(k, list(seq))
        f = _tree_form(k, e)
        if f not in seen:
            seen.add(f)
            out.append(e)
    return out


def _prufer_decode(k: int, seq) -> list[tuple[int, int]]:
    degree = [1] * k
    for x in seq:
        degree[x] += 1
    edges = []
    for x in seq:
        leaf = min(i for i in range(k) if degree[i] == 1)
        edges.append((leaf, x))
        degree[leaf] -= 1
        degree[x] -= 1
    u, w = [i for i in range(k) if degree[i] == 1]
    edges.append((u, w))
    return edges


# Tree templates used by the workloads (vertex 0..k-1).
TEMPLATES: dict[str, list[tuple[int, int]]] = {
    "P1": [],
    "P2": [(0, 1)],
    "P3": [(0, 1), (1, 2)],
    "P5": [(0, 1), (1, 2), (2, 3), (3, 4)],
    # spine 0-1-2-3-4, leaves 5,6 on 1, 7 on 2, 8,9 on 3
    "caterpillar10": [(0, 1), (1, 2), (2, 3), (3, 4), (1, 5), (1, 6), (2, 7), (3, 8), (3, 9)],
    # spine 0-1-2-3-4-5, leaves 6,7 on 1, 8 on 2, 9,10 on 4, 11 on 5
    "tree12": [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (1, 6), (1, 7), (2, 8), (4, 9), (4, 10), (5, 11)],
    # centre 0; legs 0-1-2-3, 0-4-5-6, 0-7-8-9, 0-10-11, 0-12-13, 0-14
    "spider15": [(0, 1), (1, 2), (2, 3), (0, 4), (4, 5), (5, 6), (0, 7), (7, 8), (8, 9),
                 (0, 10), (10, 11), (0, 12), (12, 13), (0, 14)],
}


def template_edges(name: str) -> tuple[int, list[tuple[int, int]]]:
    """(k, edges) of a named template."""
    e = TEMPLATES[name]
    k = 1 + max((max(x) for x in e), default=0)
    return k, list(e)
