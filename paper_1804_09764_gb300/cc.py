"""Thin Python binding of the C ABI in ``include/cc.h`` (ctypes).

Argument marshalling only: every step of the counting path runs in the CUDA
library ``_build/libcc_gb300.so``.  PyTorch supplies device memory (the arena
the library carves its buffers from) and the CUDA stream.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcc_gb300.so")

CC_OK = 0
CC_PENDING = 1
STATUS = {
    0: "CC_OK", 1: "CC_PENDING", -1: "CC_ERR_INVALID_ARG", -2: "CC_ERR_BAD_GRAPH", -3: "CC_ERR_NOT_TREE",
    -4: "CC_ERR_K_RANGE", -5: "CC_ERR_BUDGET", -6: "CC_ERR_WIDTH", -7: "CC_ERR_CUDA", -8: "CC_ERR_TIMEOUT",
    -9: "CC_ERR_CANCELLED", -10: "CC_ERR_NOT_FOUND", -11: "CC_ERR_CAPACITY", -12: "CC_ERR_NO_MEMORY",
    -13: "CC_ERR_INTERNAL",
}
CC_VALIDATE = 1
KERNEL_KINDS = 9

# names every build must export (checked by the CPU test-suite)
EXPORTED = [
    "cc_default_options", "cc_create", "cc_destroy", "cc_last_error", "cc_status_string",
    "cc_graph_load_csr", "cc_graph_free", "cc_template_load", "cc_template_free", "cc_count",
    "cc_count_ex", "cc_plan_info_get", "cc_kernel_stats_get", "cc_kernel_stats_reset", "cc_submit",
    "cc_poll", "cc_wait", "cc_cancel", "cc_serve_stats_get", "cc_template_cost",
    "cc_template_automorphisms", "cc_version", "cc_table_gather", "cc_table_gather_noalloc",
    "cc_iterations_for", "cc_estimate", "cc_count_multi", "cc_multi_plan_info_get", "cc_limb_product_rate",
    "cc_template_load_labelled", "cc_graph_set_labels", "cc_template_automorphisms_labelled",
]


class CCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class cc_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("width_bits", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("arena", ctypes.c_void_p), ("hbm_budget_bytes", ctypes.c_uint64),
                ("split_threshold", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("block_vertices", ctypes.c_int32), ("use_cuda_graph", ctypes.c_int32),
                ("fused", ctypes.c_int32), ("autotune", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("gather_mode", ctypes.c_int32), ("vertex_order", ctypes.c_int32),
                ("col_chunks", ctypes.c_int32), ("l2_persist_mb", ctypes.c_int32), ("full_rows", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 1)]


class cc_result(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("limbs", ctypes.c_int32), ("exact", ctypes.c_int32),
                ("n_iter", ctypes.c_int32), ("aut", ctypes.c_int64), ("root", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("estimate", ctypes.c_double), ("median_of_means", ctypes.c_double),
                ("device_seconds", ctypes.c_double), ("wall_seconds", ctypes.c_double),
                ("workspace_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_int64)]


class cc_multi_info(ctypes.Structure):
    _fields_ = [("chains", ctypes.c_int32), ("chains_separate", ctypes.c_int32),
                ("updates_per_colouring", ctypes.c_double), ("updates_per_colouring_separate", ctypes.c_double),
                ("workspace_bytes", ctypes.c_uint64), ("batch", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class cc_estimate_result(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("groups", ctypes.c_int32), ("n_iter", ctypes.c_int64),
                ("per_group", ctypes.c_int64), ("estimate", ctypes.c_double), ("mean", ctypes.c_double),
                ("min_group_mean", ctypes.c_double), ("max_group_mean", ctypes.c_double),
                ("device_seconds", ctypes.c_double), ("wall_seconds", ctypes.c_double)]


class cc_count_args(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("first_iter", ctypes.c_int64), ("n_iter", ctypes.c_int32),
                ("mom_groups", ctypes.c_int32), ("width_bits", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("sample_vertices", ctypes.c_void_p), ("n_sample", ctypes.c_int64),
                ("sample_maps", ctypes.c_void_p), ("maps", ctypes.c_void_p)]


class cc_plan_info(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("root", ctypes.c_int32), ("n_chains", ctypes.c_int32),
                ("n_tables", ctypes.c_int32), ("limbs_root", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("n_vertices", ctypes.c_int64), ("n_active", ctypes.c_int64),
                ("n_directed_edges", ctypes.c_int64), ("n_blocks", ctypes.c_int64),
                ("updates_per_colouring", ctypes.c_double), ("gather_bytes_per_colouring", ctypes.c_double),
                ("algorithmic_bytes_per_colouring", ctypes.c_double), ("pairs_per_colouring", ctypes.c_double),
                ("workspace_bytes", ctypes.c_uint64), ("table4_memory", ctypes.c_int64),
                ("table4_computation", ctypes.c_int64), ("limb_products_per_colouring", ctypes.c_double),
                ("split_threshold", ctypes.c_int64), ("block_vertices", ctypes.c_int64),
                ("col_chunks", ctypes.c_int32), ("shape_tuned", ctypes.c_int32),
                ("workspace_no_reuse_bytes", ctypes.c_uint64), ("workspace_no_blocks_bytes", ctypes.c_uint64),
                ("workspace_naive_bytes", ctypes.c_uint64)]


class cc_step_info(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in ("chain", "step", "vertex", "child", "h", "a", "p", "src_chain",
                                             "is_root", "limbs", "agg_limbs", "src_limbs", "chain_limbs",
                                             "path")] + [("kernel_limbs", ctypes.c_int32 * 3)]


STEP_PATHS = {0: "not_run", 1: "chain_kernel", 2: "in_chain", 3: "segmented", 4: "fused_select",
              5: "gather_select", 6: "gather_combine", 7: "leaf_select", 8: "leaf_combine"}


class cc_instance_stats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 96), ("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("timed_launches", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class cc_kernel_stats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p * KERNEL_KINDS), ("launches", ctypes.c_int64 * KERNEL_KINDS),
                ("seconds", ctypes.c_double * KERNEL_KINDS), ("bytes", ctypes.c_double * KERNEL_KINDS),
                ("total_launches", ctypes.c_int64)]


class cc_request(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int64), ("tmpl", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("first_iter", ctypes.c_int64), ("n_iter", ctypes.c_int32), ("priority", ctypes.c_int32)]


class cc_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("in_flight", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
                ("mean_latency_s", ctypes.c_double), ("busy_seconds", ctypes.c_double),
                ("admissions_deferred", ctypes.c_int64), ("passes", ctypes.c_int64),
                ("shared_passes", ctypes.c_int64), ("colourings_run", ctypes.c_int64), ("groups", ctypes.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_1804_09764_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "cc_default_options": (None, [P]),
        "cc_create": (I32, [P, P]),
        "cc_destroy": (I32, [P]),
        "cc_last_error": (ctypes.c_char_p, []),
        "cc_status_string": (ctypes.c_char_p, [I32]),
        "cc_graph_load_csr": (I32, [P, I64, P, P, ctypes.c_uint32, P]),
        "cc_graph_load_batch": (I32, [P, I32, P, I64, P, P, ctypes.c_uint32, P]),
        "cc_graph_members": (I32, [P, I64, P]),
        "cc_count_batch": (I32, [P, I64, I64, P, P, I32, P, P]),
        "cc_graph_free": (I32, [P, I64]),
        "cc_template_load": (I32, [P, I32, P, I32, P]),
        "cc_template_free": (I32, [P, I64]),
        "cc_count": (I32, [P, I64, I64, U64, I32, P, I32, P]),
        "cc_count_ex": (I32, [P, I64, I64, P, P, I32, P]),
        "cc_plan_info_get": (I32, [P, I64, I64, P]),
        "cc_kernel_stats_get": (I32, [P, P]),
        "cc_kernel_stats_reset": (I32, [P]),
        "cc_plan_steps_get": (I32, [P, I64, I64, P, I32, P]),
        "cc_kernel_instance_stats_get": (I32, [P, P, I32, P]),
        "cc_submit": (I32, [P, P, P]),
        "cc_poll": (I32, [P, I64, P, P, I32]),
        "cc_wait": (I32, [P, I64, I64, P, P, I32]),
        "cc_cancel": (I32, [P, I64]),
        "cc_serve_stats_get": (I32, [P, P]),
        "cc_template_cost": (I32, [I32, P, I32, I32, P, P]),
        "cc_template_automorphisms": (I32, [I32, P, P]),
        "cc_version": (ctypes.c_char_p, []),
        "cc_table_gather": (I32, [P, I64, P, P, P, P, I64, I32, I32]),
        "cc_table_gather_noalloc": (I32, [I64, P, P, P, P, I64, I32, I32, P]),
        "cc_iterations_for": (I32, [I32, ctypes.c_double, ctypes.c_double, P, P]),
        "cc_estimate": (I32, [P, I64, I64, U64, I64, ctypes.c_double, ctypes.c_double, I64, P]),
        "cc_count_multi": (I32, [P, I64, P, I32, P, P, I32, P]),
        "cc_multi_plan_info_get": (I32, [P, I64, P, I32, I32, P]),
        "cc_limb_product_rate": (I32, [P, P]),
        "cc_template_load_labelled": (I32, [P, I32, P, P, I32, P]),
        "cc_graph_set_labels": (I32, [P, I64, P]),
        "cc_template_automorphisms_labelled": (I32, [I32, P, P, P]),
        "cc_template_canonical_form": (I32, [I32, P, P, P, I32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status not in (CC_OK, CC_PENDING):
        raise CCError(status, _lib.cc_last_error().decode())
    return status


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def limbs_to_int(row) -> int:
    return sum(int(x) << (64 * i) for i, x in enumerate(row))


def _edges_array(k, edges):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    if e.size != 2 * (k - 1):
        raise ValueError("a tree on k vertices has k-1 edges")
    return e if e.size else np.zeros(2, dtype=np.int32)


# ------------------------------------------------------------------ host-only helpers

def cc_template_cost(k: int, edges, root: int, order: int = 0) -> tuple[int, int]:
    lib = load_library()
    mem, comp = ctypes.c_int64(), ctypes.c_int64()
    e = _edges_array(k, edges)
    _check(lib.cc_template_cost(k, _ptr(e), root, order, ctypes.byref(mem), ctypes.byref(comp)))
    return mem.value, comp.value


def cc_template_automorphisms(k: int, edges) -> int:
    lib = load_library()
    a = ctypes.c_int64()
    e = _edges_array(k, edges)
    _check(lib.cc_template_automorphisms(k, _ptr(e), ctypes.byref(a)))
    return a.value


def cc_template_automorphisms_labelled(k: int, edges, labels) -> int:
    lib = load_library()
    a = ctypes.c_int64()
    e = _edges_array(k, edges)
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8).reshape(-1))
    if lab.size != k:
        raise ValueError("one label per template vertex")
    _check(lib.cc_template_automorphisms_labelled(k, _ptr(e), _ptr(lab), ctypes.byref(a)))
    return a.value


def cc_template_canonical_form(k: int, edges, labels=None) -> str:
    """cc_template_canonical_form: equal strings exactly for isomorphic trees."""
    lib = load_library()
    lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8)
    buf = ctypes.create_string_buffer(4096)
    _check(lib.cc_template_canonical_form(k, _ptr(_edges_array(k, edges)), _ptr(lab), buf, len(buf)))
    return buf.value.decode()


def cc_iterations_for(k: int, epsilon: float, delta: float) -> tuple[int, int]:
    """(n_iter, groups) of Algorithm 1 for a (1 +- epsilon) estimate with
    probability >= 1 - delta (host only)."""
    lib = load_library()
    n, t = ctypes.c_int64(), ctypes.c_int32()
    _check(lib.cc_iterations_for(k, float(epsilon), float(delta), ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def cc_table_gather_noalloc(row_ptr, col_idx, X, agg, values: int, limbs: int, split: int = 0,
                            stream: int = 0):
    """cc_table_gather_noalloc on torch device tensors (no context, no device
    allocation by the library); returns after the gather kernels are queued on
    ``stream`` (a raw cudaStream_t handle, 0 = legacy default stream)."""
    lib = load_library()
    n = row_ptr.numel() - 1
    _check(lib.cc_table_gather_noalloc(n, row_ptr.data_ptr(), col_idx.data_ptr(), X.data_ptr(), agg.data_ptr(),
                                       values, limbs, split, stream or None))


# ------------------------------------------------------------------ context

class Context:
    """One library context on one GPU.

    ``budget_bytes``: size of the device arena (torch allocates it); every
    table and workspace of the library lives there.  Options mirror
    ``cc_options`` in include/cc.h.
    """

    def __init__(self, device: int = 0, budget_bytes: Optional[int] = None, width_bits: int = 0,
                 split_threshold: int = 0, batch: int = 0, block_vertices: int = 0, use_cuda_graph: int = 0,
                 fused: int = 1, autotune: int = 0, max_slots: int = 4, timing: int = 0, gather_mode: int = 1,
                 vertex_order: int = 0, col_chunks: int = 0, l2_persist_mb: int = 0, full_rows: int = 0, stream=None):
        import torch

        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the colour-coding library has no CPU path")
        self._lib = lib
        self.device = device
        torch.cuda.set_device(device)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(device)
            budget_bytes = int(free * 0.85)
        self._arena = torch.empty(int(budget_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        opt = cc_options()
        lib.cc_default_options(ctypes.byref(opt))
        opt.device = device
        opt.width_bits = width_bits
        opt.stream = self.stream.cuda_stream
        opt.arena = self._arena.data_ptr()
        opt.hbm_budget_bytes = int(budget_bytes)
        opt.split_threshold = split_threshold
        opt.batch = batch
        opt.block_vertices = block_vertices
        opt.use_cuda_graph = use_cuda_graph
        opt.fused = fused
        opt.autotune = autotune
        opt.max_slots = max_slots
        opt.timing = timing
        opt.gather_mode = gather_mode
        opt.vertex_order = vertex_order
        opt.col_chunks = col_chunks
        opt.l2_persist_mb = l2_persist_mb
        opt.full_rows = full_rows
        torch.cuda.synchronize(device)
        h = ctypes.c_void_p()
        _check(lib.cc_create(ctypes.byref(h), ctypes.byref(opt)))
        self._h = h

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.cc_destroy(self._h))
            self._h = None
            self._arena = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs
    def graph_load_csr(self, row_ptr, col_idx, n: Optional[int] = None, validate: bool = False) -> int:
        rp = row_ptr if hasattr(row_ptr, "data_ptr") else np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = col_idx if hasattr(col_idx, "data_ptr") else np.ascontiguousarray(col_idx, dtype=np.int32)
        if n is None:
            n = (rp.numel() if hasattr(rp, "numel") else rp.size) - 1
        gid = ctypes.c_int64()
        _check(self._lib.cc_graph_load_csr(self._h, n, _ptr(rp), _ptr(ci), CC_VALIDATE if validate else 0,
                                           ctypes.byref(gid)))
        return gid.value

    def graph_load(self, graph, validate: bool = False) -> int:
        """Load a ``graphgen.CSRGraph``."""
        return self.graph_load_csr(graph.row_ptr, graph.col_idx, graph.n, validate)

    def graph_load_batch(self, graphs, validate: bool = False) -> int:
        """cc_graph_load_batch: several ``graphgen.CSRGraph`` as one resident
        disjoint union (member i = graphs[i])."""
        off = np.zeros(len(graphs) + 1, dtype=np.int64)
        for i, g in enumerate(graphs):
            off[i + 1] = off[i] + g.n
        rp = [np.zeros(1, dtype=np.int64)]
        ci = []
        e0 = 0
        for i, g in enumerate(graphs):
            rp.append(np.asarray(g.row_ptr[1:], dtype=np.int64) + e0)
            ci.append(np.asarray(g.col_idx, dtype=np.int64) + off[i])
            e0 += int(g.row_ptr[-1])
        rp = np.concatenate(rp)
        ci = np.concatenate(ci).astype(np.int32) if ci else np.zeros(0, np.int32)
        return self.graph_load_batch_csr(off, rp, ci, validate)

    def graph_load_batch_csr(self, member_off, row_ptr, col_idx, validate: bool = False) -> int:
        """cc_graph_load_batch on the union's CSR arrays (host)."""
        off = np.ascontiguousarray(member_off, dtype=np.int64)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        gid = ctypes.c_int64()
        _check(self._lib.cc_graph_load_batch(self._h, off.size - 1, _ptr(off), int(off[-1]), _ptr(rp), _ptr(ci),
                                             CC_VALIDATE if validate else 0, ctypes.byref(gid)))
        return gid.value

    def graph_members(self, gid: int) -> int:
        n = ctypes.c_int32()
        _check(self._lib.cc_graph_members(self._h, gid, ctypes.byref(n)))
        return n.value

    def graph_free(self, gid: int):
        _check(self._lib.cc_graph_free(self._h, gid))

    def template_load(self, k: int, edges, root: int = -1, labels=None) -> int:
        """cc_template_load, or cc_template_load_labelled with k vertex labels."""
        tid = ctypes.c_int64()
        e = _edges_array(k, edges)
        if labels is None:
            _check(self._lib.cc_template_load(self._h, k, _ptr(e), root, ctypes.byref(tid)))
        else:
            lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8).reshape(-1))
            if lab.size != k:
                raise ValueError("one label per template vertex")
            _check(self._lib.cc_template_load_labelled(self._h, k, _ptr(e), _ptr(lab), root, ctypes.byref(tid)))
        return tid.value

    def graph_set_labels(self, gid: int, labels):
        """cc_graph_set_labels: one uint8 label per vertex (None removes them)."""
        if labels is None:
            _check(self._lib.cc_graph_set_labels(self._h, gid, None))
            return
        lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8).reshape(-1))
        _check(self._lib.cc_graph_set_labels(self._h, gid, _ptr(lab)))

    def template_free(self, tid: int):
        _check(self._lib.cc_template_free(self._h, tid))

    # -- counting
    def count(self, gid: int, tid: int, seed: int, n_iter: int, first_iter: int = 0, limbs_capacity: int = 4,
              width_bits: int = -1, mom_groups: int = 1, sample_vertices: Optional[Sequence[int]] = None,
              want_maps: bool = False, raw: bool = False):
        """cc_count_ex.  Returns a dict with per-colouring counts as Python ints
        (or the raw uint64 limb arrays with ``raw=True``) and the result fields."""
        cap = limbs_capacity
        counts = np.zeros((max(n_iter, 1), cap), dtype=np.uint64)
        maps = np.zeros((max(n_iter, 1), cap), dtype=np.uint64) if want_maps else None
        args = cc_count_args()
        args.seed = seed & (2 ** 64 - 1)
        args.first_iter = first_iter
        args.n_iter = n_iter
        args.mom_groups = mom_groups
        args.width_bits = width_bits
        sv = smaps = None
        if sample_vertices is not None and len(sample_vertices):
            sv = np.ascontiguousarray(np.asarray(sample_vertices, dtype=np.int64))
            smaps = np.zeros((max(n_iter, 1), sv.size, cap), dtype=np.uint64)
            args.sample_vertices = sv.ctypes.data
            args.n_sample = sv.size
            args.sample_maps = smaps.ctypes.data
        if maps is not None:
            args.maps = maps.ctypes.data
        res = cc_result()
        _check(self._lib.cc_count_ex(self._h, gid, tid, ctypes.byref(args), _ptr(counts), cap, ctypes.byref(res)))
        out = {f: getattr(res, f) for f, _ in cc_result._fields_}
        if raw:
            out["counts_raw"] = counts[:n_iter]
            out["maps_raw"] = None if maps is None else maps[:n_iter]
            out["samples_raw"] = None if smaps is None else smaps[:n_iter]
        out["counts"] = [limbs_to_int(r) for r in counts[:n_iter]]
        if maps is not None:
            out["maps"] = [limbs_to_int(r) for r in maps[:n_iter]]
        if smaps is not None:
            out["samples"] = [[limbs_to_int(r) for r in smaps[j]] for j in range(n_iter)]
        return out

    def count_batch(self, gid: int, tid: int, seed: int, n_iter: int, first_iter: int = 0,
                    limbs_capacity: int = 4, width_bits: int = -1, want_maps: bool = False) -> dict:
        """cc_count_batch: per member graph counts (``counts[i]`` = member i's
        per-colouring counts, ``estimates[i]`` its estimate) and the shared
        result fields."""
        cap = limbs_capacity
        m = self.graph_members(gid)
        counts = np.zeros((m, max(n_iter, 1), cap), dtype=np.uint64)
        maps = np.zeros((m, max(n_iter, 1), cap), dtype=np.uint64) if want_maps else None
        est = np.zeros(m, dtype=np.float64)
        args = cc_count_args()
        args.seed = seed & (2 ** 64 - 1)
        args.first_iter = first_iter
        args.n_iter = n_iter
        args.mom_groups = 1
        args.width_bits = width_bits
        if maps is not None:
            args.maps = maps.ctypes.data
        res = cc_result()
        _check(self._lib.cc_count_batch(self._h, gid, tid, ctypes.byref(args), _ptr(counts), cap, _ptr(est),
                                        ctypes.byref(res)))
        out = {f: getattr(res, f) for f, _ in cc_result._fields_}
        out["counts"] = [[limbs_to_int(r) for r in counts[i, :n_iter]] for i in range(m)]
        if maps is not None:
            out["maps"] = [[limbs_to_int(r) for r in maps[i, :n_iter]] for i in range(m)]
        out["estimates"] = est.tolist()
        return out

    def count_multi(self, gid: int, tids: Sequence[int], seed: int, n_iter: int, first_iter: int = 0,
                    limbs_capacity: int = 4, width_bits: int = -1, mom_groups: int = 1,
                    want_maps: bool = False) -> list:
        """cc_count_multi: one result dict per template (as ``count``)."""
        cap, nt = limbs_capacity, len(tids)
        ids = np.ascontiguousarray(np.asarray(tids, dtype=np.int64))
        counts = np.zeros((nt, max(n_iter, 1), cap), dtype=np.uint64)
        maps = np.zeros((nt, max(n_iter, 1), cap), dtype=np.uint64) if want_maps else None
        args = cc_count_args()
        args.seed = seed & (2 ** 64 - 1)
        args.first_iter = first_iter
        args.n_iter = n_iter
        args.mom_groups = mom_groups
        args.width_bits = width_bits
        if maps is not None:
            args.maps = maps.ctypes.data
        res = (cc_result * max(nt, 1))()
        _check(self._lib.cc_count_multi(self._h, gid, _ptr(ids), nt, ctypes.byref(args), _ptr(counts), cap, res))
        out = []
        for r in range(nt):
            d = {f: getattr(res[r], f) for f, _ in cc_result._fields_}
            d["counts"] = [limbs_to_int(x) for x in counts[r, :n_iter]]
            if maps is not None:
                d["maps"] = [limbs_to_int(x) for x in maps[r, :n_iter]]
            out.append(d)
        return out

    def multi_plan_info(self, gid: int, tids: Sequence[int], n_iter: int = 1) -> dict:
        ids = np.ascontiguousarray(np.asarray(tids, dtype=np.int64))
        info = cc_multi_info()
        _check(self._lib.cc_multi_plan_info_get(self._h, gid, _ptr(ids), len(tids), n_iter, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in cc_multi_info._fields_}

    def plan_info(self, gid: int, tid: int) -> dict:
        info = cc_plan_info()
        _check(self._lib.cc_plan_info_get(self._h, gid, tid, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in cc_plan_info._fields_}

    def plan_steps(self, gid: int, tid: int) -> list:
        """cc_plan_steps_get: one dict per DP step (widths and the path the last pass took)."""
        n = ctypes.c_int32()
        _check(self._lib.cc_plan_steps_get(self._h, gid, tid, None, 0, ctypes.byref(n)))
        arr = (cc_step_info * max(1, n.value))()
        _check(self._lib.cc_plan_steps_get(self._h, gid, tid, arr, n.value, ctypes.byref(n)))
        out = []
        for r in arr[:n.value]:
            d = {f: getattr(r, f) for f, _ in cc_step_info._fields_ if f != "kernel_limbs"}
            d["kernel_limbs"] = tuple(r.kernel_limbs)
            d["path"] = STEP_PATHS.get(d["path"], str(d["path"]))
            out.append(d)
        return out

    def kernel_instances(self) -> dict:
        """cc_kernel_instance_stats_get: {kind name: {instantiation: stats}}."""
        names = [n for n in self.kernel_stats() if n != "total_launches"]
        n = ctypes.c_int32()
        _check(self._lib.cc_kernel_instance_stats_get(self._h, None, 0, ctypes.byref(n)))
        arr = (cc_instance_stats * max(1, n.value))()
        _check(self._lib.cc_kernel_instance_stats_get(self._h, arr, n.value, ctypes.byref(n)))
        out = {nm: {} for nm in names}
        for r in arr[:n.value]:
            out[names[r.kind]][r.name.decode()] = dict(launches=r.launches, timed_launches=r.timed_launches,
                                                       seconds=r.seconds, bytes=r.bytes)
        return out

    def kernel_stats(self) -> dict:
        s = cc_kernel_stats()
        _check(self._lib.cc_kernel_stats_get(self._h, ctypes.byref(s)))
        out = {}
        for i in range(KERNEL_KINDS):
            nm = s.name[i].decode() if s.name[i] else str(i)
            out[nm] = dict(launches=s.launches[i], seconds=s.seconds[i], bytes=s.bytes[i])
        out["total_launches"] = s.total_launches
        return out

    def estimate(self, gid: int, tid: int, seed: int, epsilon: float, delta: float, first_iter: int = 0,
                 max_iter: int = 0) -> dict:
        """cc_estimate: Algorithm 1 end to end (median of group means)."""
        r = cc_estimate_result()
        _check(self._lib.cc_estimate(self._h, gid, tid, seed & (2 ** 64 - 1), first_iter, float(epsilon),
                                     float(delta), max_iter, ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in cc_estimate_result._fields_}

    def limb_product_rate(self) -> float:
        """cc_limb_product_rate: 64-bit limb products per second on this GPU."""
        r = ctypes.c_double()
        _check(self._lib.cc_limb_product_rate(self._h, ctypes.byref(r)))
        return r.value

    def kernel_stats_reset(self):
        _check(self._lib.cc_kernel_stats_reset(self._h))

    def table_gather(self, row_ptr, col_idx, X, agg, values: int, limbs: int, split: int = 0):
        """cc_table_gather on torch device tensors (row_ptr int64, col_idx int32,
        X / agg uint64-compatible int64 tensors of n*values*limbs)."""
        n = row_ptr.numel() - 1
        _check(self._lib.cc_table_gather(self._h, n, row_ptr.data_ptr(), col_idx.data_ptr(), X.data_ptr(),
                                         agg.data_ptr(), values, limbs, split))

    # -- serving
    def submit(self, gid: int, tid: int, seed: int, n_iter: int, first_iter: int = 0) -> int:
        r = cc_request(graph=gid, tmpl=tid, seed=seed & (2 ** 64 - 1), first_iter=first_iter, n_iter=n_iter)
        rid = ctypes.c_int64()
        _check(self._lib.cc_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        return rid.value

    def _result(self, status, res, counts, n_iter):
        out = {f: getattr(res, f) for f, _ in cc_result._fields_}
        out["counts"] = [limbs_to_int(r) for r in counts[:n_iter]]
        return out

    def poll(self, rid: int, n_iter: int, limbs_capacity: int = 4):
        res = cc_result()
        counts = np.zeros((max(n_iter, 1), limbs_capacity), dtype=np.uint64)
        st = _check(self._lib.cc_poll(self._h, rid, ctypes.byref(res), _ptr(counts), limbs_capacity))
        if st == CC_PENDING:
            return None
        return self._result(st, res, counts, n_iter)

    def wait(self, rid: int, n_iter: int, timeout_s: float = -1, limbs_capacity: int = 4):
        res = cc_result()
        counts = np.zeros((max(n_iter, 1), limbs_capacity), dtype=np.uint64)
        tns = -1 if timeout_s < 0 else int(timeout_s * 1e9)
        st = _check(self._lib.cc_wait(self._h, rid, tns, ctypes.byref(res), _ptr(counts), limbs_capacity))
        return self._result(st, res, counts, n_iter)

    def cancel(self, rid: int):
        _check(self._lib.cc_cancel(self._h, rid))

    def serve_stats(self) -> dict:
        s = cc_serve_stats()
        _check(self._lib.cc_serve_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in cc_serve_stats._fields_}
