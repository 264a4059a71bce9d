"""CPU oracle for the colour-coding tree counter (arXiv 1804.09764, Section 2.1).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the package's smoke
check and by the benchmark's CPU-baseline / reference leg.  The product path
never imports it.  It shares no code with the CUDA path; the only module both
use is the seeded input generator (``paper_1804_09764_gb300.graphgen``), which
holds no arithmetic of the method.

``count`` wraps the C implementation in ``cc_oracle.c`` (Eq. 1 written out
with d = 1, exact modulo 2^256).  The host-side finishing steps of Algorithm 1
live here in plain Python integers:
  * copies_j = maps_j / |Aut(T)| (exact division, Section 2.1: an embedding is
    reached once per automorphism when d = 1),
  * est_j = copies_j * k^k / k!                        (Eq. 3),
  * median of means over t equal groups                (Algorithm 1, last step).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcc_oracle.so")
_lib = None

MOD256 = 1 << 256


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vector intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.cco_count.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int, P, ctypes.c_int,
                                  ctypes.c_uint64, ctypes.c_uint64, P, P, P, P]
        lib.cco_count.restype = ctypes.c_int
        lib.cco_automorphisms.argtypes = [ctypes.c_int, P]
        lib.cco_automorphisms.restype = ctypes.c_int64
        lib.cco_automorphisms_labelled.argtypes = [ctypes.c_int, P, P]
        lib.cco_automorphisms_labelled.restype = ctypes.c_int64
        lib.cco_colour.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
        lib.cco_colour.restype = ctypes.c_int
        lib.cco_splitmix64.argtypes = [ctypes.c_uint64]
        lib.cco_splitmix64.restype = ctypes.c_uint64
        for f in (lib.cco_u256_mul, lib.cco_u256_add):
            f.argtypes = [P, P, P]
            f.restype = None
        _lib = lib
    return _lib


def _limbs_to_int(a) -> int:
    return sum(int(x) << (64 * i) for i, x in enumerate(a))


def _int_to_limbs(x: int) -> np.ndarray:
    return np.array([(x >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _edges_array(k, edges):
    e = np.asarray(edges, dtype=np.int32).reshape(-1)
    if e.size != 2 * (k - 1):
        raise ValueError("a tree on k vertices has k-1 edges")
    return np.ascontiguousarray(e) if e.size else np.zeros(2, dtype=np.int32)


def automorphisms(k: int, edges, labels=None) -> int:
    """|Aut(T)| by backtracking over bijections of V_T (with labels: only the
    label-preserving ones)."""
    if labels is not None:
        lab = np.ascontiguousarray(labels, dtype=np.uint8)
        r = _load().cco_automorphisms_labelled(k, _ptr(_edges_array(k, edges)), _ptr(lab))
    else:
        r = _load().cco_automorphisms(k, _ptr(_edges_array(k, edges)))
    if r < 0:
        raise ValueError("template is not a tree")
    return int(r)


def colour(seed: int, j: int, ids, k: int) -> np.ndarray:
    """Colours of the given vertex ids for colouring j (uint8)."""
    lib = _load()
    return np.array([lib.cco_colour(seed, j, int(i), k) for i in np.asarray(ids).reshape(-1)],
                    dtype=np.uint8)


def splitmix64(state: int) -> int:
    return int(_load().cco_splitmix64(state))


def u256_mul(a: int, b: int) -> int:
    r = np.zeros(4, dtype=np.uint64)
    _load().cco_u256_mul(_ptr(_int_to_limbs(a)), _ptr(_int_to_limbs(b)), _ptr(r))
    return _limbs_to_int(r)


def u256_add(a: int, b: int) -> int:
    r = np.zeros(4, dtype=np.uint64)
    _load().cco_u256_add(_ptr(_int_to_limbs(a)), _ptr(_int_to_limbs(b)), _ptr(r))
    return _limbs_to_int(r)


def count_maps(graph, k: int, edges, root: int = 0, seed: int = 0, j: int = 0,
               colours=None, ids=None, per_vertex: bool = False, glabels=None, tlabels=None):
    """Colourful maps (injective homomorphisms V_T -> V_G whose images have k
    distinct colours) for colouring j, mod 2^256.  With vertex labels glabels
    [n] and tlabels [k] (both or neither) only label-preserving maps count.

    Returns ``maps`` or ``(maps, per_vertex_list)``.
    """
    lib = _load()
    n = graph.n
    rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(graph.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    col = None if colours is None else np.ascontiguousarray(colours, dtype=np.uint8)
    idv = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    tot = np.zeros(4, dtype=np.uint64)
    pv = np.zeros((max(n, 1), 4), dtype=np.uint64) if per_vertex else None
    gl = None if glabels is None else np.ascontiguousarray(glabels, dtype=np.uint8)
    tl = None if tlabels is None else np.ascontiguousarray(tlabels, dtype=np.uint8)
    if (gl is None) != (tl is None) or (gl is not None and (gl.size != n or tl.size != k)):
        raise ValueError("give graph and template labels together, one per vertex")
    rc = lib.cco_count(n, _ptr(rp), _ptr(ci), _ptr(idv), _ptr(col), k,
                       _ptr(_edges_array(k, edges)), root, seed & (2**64 - 1), j, _ptr(tot), _ptr(pv),
                       _ptr(gl), _ptr(tl))
    if rc != 0:
        raise RuntimeError(f"oracle failed: {rc}")
    maps = _limbs_to_int(tot)
    if per_vertex:
        return maps, [_limbs_to_int(pv[v]) for v in range(n)]
    return maps


def copies_from_maps(maps: int, aut: int) -> int:
    """copies = maps / |Aut(T)|; exact (maps must be the true count < 2^256)."""
    q, r = divmod(maps, aut)
    if r:
        raise ArithmeticError("maps not divisible by |Aut(T)|")
    return q


def estimate(copies: int, k: int) -> float:
    """Eq. 3: C^(j) = k^k / k! * (colourful copies)."""
    return float(Fraction(copies * k ** k, math.factorial(k)))


def median_of_means(estimates, t: int) -> float:
    """Algorithm 1, last step: split into t sets of equal size q = N // t
    (the first t*q estimates, in order), average each, take the median."""
    est = list(estimates)
    if t < 1 or t > len(est):
        raise ValueError("need 1 <= t <= number of estimates")
    q = len(est) // t
    means = sorted(math.fsum(est[g * q:(g + 1) * q]) / q for g in range(t))
    if t % 2:
        return means[t // 2]
    return 0.5 * (means[t // 2 - 1] + means[t // 2])


def neighbour_sum(graph, X: np.ndarray, limbs: int) -> np.ndarray:
    """Eq. 1's inner sum over u in N(v) of a count table, on its own:
    out[v] = sum_{u in N(v)} X[u], each value an integer of `limbs` 64-bit limbs
    (least significant first) added modulo 2^(64*limbs).  X: uint64
    [n][values][limbs]; plain Python integers."""
    n, values, L = X.shape
    assert L == limbs
    M = 1 << (64 * limbs)
    vals = [[sum(int(X[u, c, i]) << (64 * i) for i in range(L)) for c in range(values)] for u in range(n)]
    out = np.zeros_like(X)
    for v in range(n):
        acc = [0] * values
        for u in graph.neighbours(v):
            row = vals[int(u)]
            for c in range(values):
                acc[c] += row[c]
        for c in range(values):
            x = acc[c] % M
            for i in range(L):
                out[v, c, i] = (x >> (64 * i)) & ((1 << 64) - 1)
    return out


def run(graph, k: int, edges, seed: int, n_iter: int, root: int = 0, first_iter: int = 0):
    """Algorithm 1 for colourings first_iter .. first_iter+n_iter-1.

    Returns dict(maps=[...], copies=[...], estimates=[...], aut=..., mean=...).
    """
    aut = automorphisms(k, edges)
    maps = [count_maps(graph, k, edges, root, seed, first_iter + j) for j in range(n_iter)]
    copies = [copies_from_maps(m, aut) for m in maps]
    ests = [estimate(c, k) for c in copies]
    return dict(maps=maps, copies=copies, estimates=ests, aut=aut,
                mean=math.fsum(ests) / len(ests) if ests else 0.0)
