"""Writes tree12_widths.json: oracle counts for the tree-12 template on a graph
whose homomorphism bounds give the same integer widths per kernel as R-MAT
scale 22 does (Eq. 1 tables of 1 limb for the 66-, 792- and 924-column
tables, 2 limbs for the 495-column table and for the root chain's gather
step, 3 limbs for the root chain's leaf steps and total), but small enough for
the oracle.

The graph is the disjoint union of K_{500,6000} and R-MAT scale 11 (seed 11):
the 500 vertices of degree 6000 exceed the 4096-neighbour task size
(Algorithm 4's split), the 6000 of degree 500 and the R-MAT vertices are
light.  With c = 500 and N = 6000 the rooted homomorphism bounds are, in
bits: 924-column table c^2 N^3 ~ 55.6; the 495-column chain's gather
c^2 N^4 ~ 68.1 and its table c^2 N^5 ~ 80.7; the root chain's gather
c^3 N^5 ~ 89.7; the root total 2 c^6 N^6 ~ 130.1.

Run from the repository root:  python tests/golden/make_tree12_widths.py
It calls only the seeded generators and the oracle (about 90 s per colouring).
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1804_09764_gb300 import graphgen as gg  # noqa: E402

C_HUBS, N_LEAVES, RMAT_SCALE = 500, 6000, 11
SEED, COLOURINGS, ROOT_VERTEX = 2222, (0, 1), 1


def graph():
    return gg.disjoint_union(gg.complete_bipartite_graph(C_HUBS, N_LEAVES), gg.rmat_graph(RMAT_SCALE, seed=RMAT_SCALE))


def digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(g.col_idx, dtype=np.int32).tobytes())
    return h.hexdigest()


def sample_vertices(g):
    """Every 10th degree-N vertex, every 100th degree-c vertex, every 20th
    R-MAT vertex and the 20 R-MAT vertices of highest degree."""
    hubs = list(range(0, C_HUBS, 10))
    leaves = list(range(C_HUBS, C_HUBS + N_LEAVES, 100))
    base = C_HUBS + N_LEAVES
    core = list(range(base, g.n, 20))
    deg = np.diff(g.row_ptr)[base:]
    top = [base + int(v) for v in np.argsort(-deg, kind="stable")[:20]]
    return sorted(set(hubs + leaves + core + top + [g.n - 1]))


def main():
    g = graph()
    k, e = gg.template_edges("tree12")
    sample = sample_vertices(g)
    out = {"template": "tree12", "k": k, "root": ROOT_VERTEX, "seed": SEED, "colourings": list(COLOURINGS),
           "graph": {"recipe": f"disjoint_union(complete_bipartite_graph({C_HUBS}, {N_LEAVES}), "
                               f"rmat_graph({RMAT_SCALE}, seed={RMAT_SCALE}))",
                     "n": g.n, "nnz": g.nnz, "sha256": digest(g)},
           "aut": O.automorphisms(k, e), "maps": [], "sample_vertices": sample, "sample_maps": []}
    for j in COLOURINGS:
        t = time.time()
        m, pv = O.count_maps(g, k, e, ROOT_VERTEX, seed=SEED, j=j, per_vertex=True)
        out["maps"].append(hex(m))
        out["sample_maps"].append([hex(pv[v]) for v in sample])
        print(f"colouring {j}: {m.bit_length()} bits, {time.time() - t:.1f} s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tree12_widths.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
