"""Benchmark of the colour-coding tree counter on one GB300 (or N replicas).

One step = one pass of the whole hot path (colour, leaf gather, table gathers,
combines, root reduce, host finish) over the workload's batch of colourings.

Metric: edge x colour-set updates per second,
    U = sum over gathered non-leaf passive tables of 2m * C(k, |T_p|)
per colouring (the gather work of Eq. 1), times colourings, over device time.

Default workload: R-MAT scale 22 (a,b,c,d = .57,.19,.19,.05, edge factor 16,
seed 22, labels permuted), 12-vertex tree template, k = 12, 16 colourings,
100 GB HBM budget.

--impl reference runs the CPU oracle (the plain single-threaded DP) on a
bounded sample of the same workload on the host cores.

Under torchrun each rank runs an independent replica on its own colourings
(the colourings are independent units): no collective on the data path,
weak scaling, value = all ranks' updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1804_09764_gb300 import graphgen as gg  # noqa: E402

WORKLOADS = {
    "er2000_p5": dict(graph=("er", 2000, 8, 1), template="P5", root=2, n_iter=1, budget=4 << 30),
    "rmat20_caterpillar10": dict(graph=("rmat", 20, 20), template="caterpillar10", root=2, n_iter=64,
                                 budget=100 << 30),
    "rmat22_tree12": dict(graph=("rmat", 22, 22), template="tree12", root=-1, n_iter=16, budget=100 << 30),
    "rmat24_spider15": dict(graph=("rmat", 24, 24), template="spider15", root=0, n_iter=4, budget=150 << 30),
}
DEFAULT = "rmat22_tree12"


def make_graph(spec):
    if spec[0] == "er":
        return gg.er_graph(spec[1], spec[2], seed=spec[3])
    return gg.rmat_graph(spec[1], seed=spec[2])


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks during the timed region."""

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.device), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                f = [x.strip() for x in out.split(",")]
                if len(f) >= 7:
                    self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_sample(wl, target_s=15.0, max_scale=None):
    """Time the CPU oracle on the workload's template over R-MAT graphs of
    growing scale (same generator parameters) until one colouring takes at
    least target_s / 4; returns (updates/s, description, cores)."""
    import oracle as O

    k, e = gg.template_edges(wl["template"])
    root = wl["root"] if wl["root"] >= 0 else 0
    spec = wl["graph"]
    if spec[0] == "er":
        g = make_graph(spec)
        t = time.perf_counter()
        O.count_maps(g, k, e, root, seed=1, j=0)
        dt = time.perf_counter() - t
        return None, dt, f"oracle on the full workload ({g.n} vertices, one colouring)", g, k, e, root
    top = spec[1] if max_scale is None else min(spec[1], max_scale)
    best = None
    for s in range(8, top + 1):
        g = gg.rmat_graph(s, seed=spec[2])
        t = time.perf_counter()
        O.count_maps(g, k, e, root, seed=1, j=0)
        dt = time.perf_counter() - t
        best = (s, g, dt)
        if dt >= target_s / 4:
            break
    s, g, dt = best
    return s, dt, f"oracle, one colouring of {wl['template']} on R-MAT scale {s} (same a,b,c,d, edge factor 16)", \
        g, k, e, root


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    s, dt, desc, g, k, e, root = oracle_sample(wl, target_s=args.ref_seconds)
    U = plan_updates_host(g, k, e, root)
    steps = []
    import oracle as O
    for i in range(args.steps):
        t = time.perf_counter()
        O.count_maps(g, k, e, root, seed=1, j=i + 1)
        steps.append(time.perf_counter() - t)
    tot = sum(steps)
    value = U * len(steps) / tot
    line = {"impl": "reference", "metric": "edge_colourset_updates_per_s", "value": value,
            "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u256", "data": "synthetic",
            "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def plan_updates_host(g, k, e, root):
    """U per colouring for a graph, from the template structure only:
    sum over distinct rooted subtrees T_c (c a non-leaf, non-root vertex) of
    2m * C(k, |T_c|) — the same count the library reports."""
    adj = {i: [] for i in range(k)}
    for a, b in e:
        adj[a].append(b)
        adj[b].append(a)
    canon, size = {}, {}

    def dfs(x, p):
        cs = []
        size[x] = 1
        for y in adj[x]:
            if y != p:
                dfs(y, x)
                cs.append(canon[y])
                size[x] += size[y]
        canon[x] = "(" + "".join(sorted(cs)) + ")"

    dfs(root, -1)
    seen = set()
    U = 0
    for x in range(k):
        if x == root or size[x] == 1 or canon[x] in seen:
            continue
        seen.add(canon[x])
        U += g.nnz * math.comb(k, size[x])
    return U


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=list(WORKLOADS))
    ap.add_argument("--n-iter", type=int, default=0, help="colourings per step (0: workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.n_iter:
        wl["n_iter"] = args.n_iter
    rank, world, local = dist_env()

    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    import torch

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local)
    t0 = time.time()
    g = make_graph(wl["graph"])
    gen_s = time.time() - t0
    k, e = gg.template_edges(wl["template"])
    budget = min(wl["budget"], int(torch.cuda.mem_get_info(local)[0] * 0.9))
    ctx = cc.Context(device=local, budget_bytes=budget, timing=1, split_threshold=args.split, batch=args.batch,
                     block_vertices=args.block)
    gid = ctx.graph_load(g)
    tid = ctx.template_load(k, e, wl["root"])
    info = ctx.plan_info(gid, tid)
    n_iter = wl["n_iter"]

    def step(i):
        return ctx.count(gid, tid, seed=12345, n_iter=n_iter, first_iter=(rank * 1000 + i) * n_iter)

    for i in range(args.warmup):
        step(i)
    ctx.kernel_stats_reset()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    dev_s = 0.0
    launches = 0
    with ClockSampler(local) as clk:
        t_start = time.perf_counter()
        for i in range(args.steps):
            r = step(args.warmup + i)
            dev_s += r["device_seconds"]
            launches += r["kernel_launches"]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_start
    ks = ctx.kernel_stats()
    elapsed = dev_s
    if world > 1:
        t = torch.tensor([elapsed], dtype=torch.float64, device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
    U = info["updates_per_colouring"] * n_iter * args.steps * world
    value = U / elapsed

    # end to end through the C ABI from pinned host buffers: graph upload + count + results
    e2e = None
    if not args.no_e2e:
        rp = torch.from_numpy(g.row_ptr).pin_memory()
        ci = torch.from_numpy(g.col_idx).pin_memory()
        ctx2_t = []
        for i in range(1 + args.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            gid2 = ctx.graph_load_csr(rp, ci, g.n)
            r = ctx.count(gid2, tid, seed=777, n_iter=n_iter, first_iter=i * n_iter)
            ctx.graph_free(gid2)
            ctx2_t.append(time.perf_counter() - t)
        et = sum(ctx2_t[1:])
        e2e = {"value": info["updates_per_colouring"] * n_iter * args.steps * world / et, "unit": "updates/s",
               "h2d_bytes_per_step": int(rp.numel() * 8 + ci.numel() * 4),
               "d2h_bytes_per_step": int(n_iter * 4 * 8)}

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return
    peak, peak_kind = measured_peaks()
    kinds = {k_: v for k_, v in ks.items() if isinstance(v, dict) and v["launches"] > 0}
    dom = max(kinds.items(), key=lambda kv: kv[1]["seconds"])
    dname, d = dom
    achieved = d["bytes"] / d["seconds"] / 1e9 if d["seconds"] > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                "launches": d["launches"], "avg_launch_ms": 1e3 * d["seconds"] / d["launches"],
                "share_of_kernel_time": d["seconds"] / sum(v["seconds"] for v in kinds.values())}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        s, dt, desc, gs, k2, e2, root2 = oracle_sample(wl, target_s=15.0)
        Us = plan_updates_host(gs, k2, e2, root2)
        cpu = {"value": Us / dt, "unit": "updates/s", "cores": 1, "kind": "oracle",
               "sample": desc + f", {dt:.1f} s"}
    line = {
        "metric": "edge_colourset_updates_per_s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64/u128/u192",
        "data": "synthetic",
        "config": {"workload": args.workload, "graph": g.name, "n": g.n, "m": g.m, "n_active": info["n_active"],
                   "template": wl["template"], "k": k, "root": info["root"], "colourings_per_step": n_iter,
                   "batch": info["batch"], "blocks": info["n_blocks"], "limbs_root": info["limbs_root"],
                   "workspace_gb": info["workspace_bytes"] / 1e9, "l2": "inputs larger than L2",
                   "updates_per_colouring": info["updates_per_colouring"],
                   "algorithmic_bytes_per_colouring": info["algorithmic_bytes_per_colouring"],
                   "graph_gen_s": round(gen_s, 1), "wall_s": round(wall, 3)},
        "hbm_frac_step": info["algorithmic_bytes_per_colouring"] * n_iter * args.steps / elapsed / 1e9 / peak,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "kernels": {k_: {"launches": v["launches"], "ms": round(1e3 * v["seconds"], 3),
                         "GBps": (v["bytes"] / v["seconds"] / 1e9) if v["seconds"] else None}
                    for k_, v in kinds.items()},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.barrier()


if __name__ == "__main__":
    main()
