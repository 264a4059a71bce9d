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
    # small case of the same kernels for profiler captures (tables ~4 GB, above L2;
    # root 1, the planner's root for the scale-22 headline)
    "rmat18_tree12": dict(graph=("rmat", 18, 18), template="tree12", root=1, n_iter=1, budget=16 << 30),
    # smaller still, for full-section captures (tables ~2 GB, one vertex block)
    "rmat17_tree12": dict(graph=("rmat", 17, 17), template="tree12", root=1, n_iter=1, budget=8 << 30),
    "rmat24_spider15": dict(graph=("rmat", 24, 24), template="spider15", root=0, n_iter=4, budget=150 << 30),
    # labelled templates: 4 seeded labels on graph and template vertices
    "rmat22_tree12_labelled": dict(graph=("rmat", 22, 22), template="tree12", root=-1, n_iter=16,
                                   budget=100 << 30, labels=4),
    # small case of the spider-15 combine for profiler captures (a few GB)
    "rmat16_spider15": dict(graph=("rmat", 16, 16), template="spider15", root=0, n_iter=1, budget=6 << 30),
}
DEFAULT = "rmat22_tree12"


def make_graph(spec):
    if spec[0] == "er":
        return gg.er_graph(spec[1], spec[2], seed=spec[3])
    return gg.rmat_graph(spec[1], seed=spec[2])


def replica_first_iter(rank: int, world: int, step: int, n_iter: int) -> int:
    """Colourings are independent units (Algorithm 1's outer loop), so replicas
    shard them: step `step` of rank `rank` runs colourings
    [(step * world + rank) * n_iter, ... + n_iter) -- disjoint across ranks and
    steps, no data exchange."""
    return (step * world + rank) * n_iter


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank time over all ranks (the job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_check(per_rank, recount, rank0=0):
    """Cross-check of colouring replicas: per_rank[r] is rank r's list of
    (colouring index, count) pairs.  Colourings are independent and counts
    exact, so a count must not depend on the rank that computed it: rank 0
    recounts the first colouring of every other rank (recount(j) -> count) and
    compares.  Returns {"checked": n, "equal": bool, "colourings": total}."""
    checked, equal = 0, True
    for r, pairs in enumerate(per_rank):
        if r == rank0 or not pairs:
            continue
        j, cnt = pairs[0]
        checked += 1
        equal &= recount(j) == cnt
    return {"checked": checked, "equal": bool(equal), "colourings": sum(len(p) for p in per_rank)}


def kernel_source_digest() -> str:
    """Digest of the CUDA sources and of the planner/executor; DRAM-traffic
    figures taken with ncu are only used while these are unchanged."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1804_09764_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):  # kernels, and the planner/executor that decide their launches
        if name.endswith((".cu", ".cuh")) or name in ("exec.cpp", "plan.cpp"):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def instance_file_name(name: str) -> str:
    """File-name form of a kernel instantiation: gather_select_chain_kernel<2,2,3>
    -> gather_select_chain_kernel_2_2_3."""
    return name.replace("<", "_").replace(",", "_").replace(">", "")


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of the kernel instantiation `kernel` on `workload`
    from a committed ncu summary (profiles/traffic_<kernel>_<workload>.json), or
    None when absent or taken on different kernel sources."""
    p = os.path.join(ROOT, "profiles", f"traffic_{instance_file_name(kernel)}_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_digest") != kernel_source_digest():
        return None
    return d.get("dram_bytes_per_launch")


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


_WORKER_GRAPHS = {}


def _oracle_colouring(spec, k, e, root, seed, j):
    """One oracle colouring in a worker process (imports oracle there; the
    graph is generated once per process, outside the timed calls)."""
    import oracle as O

    if spec not in _WORKER_GRAPHS:
        _WORKER_GRAPHS[spec] = make_graph(spec)
    t = time.perf_counter()
    O.count_maps(_WORKER_GRAPHS[spec], k, e, root, seed=seed, j=j)
    return time.perf_counter() - t


def oracle_cores_rate(g_spec, k, e, root, U_per_colouring, colourings, cores):
    """The oracle on the host's cores: independent colourings (Algorithm 1's
    outer loop) in `cores` single-threaded worker processes, started with
    spawn (a process forked after CUDA initialisation would hang).  Returns
    (updates/s over the wall time of the batch, wall seconds)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_colouring, [g_spec] * cores, [k] * cores, [e] * cores, [root] * cores,
                    [1] * cores, range(1000, 1000 + cores)))  # start-up and graph build, untimed
        t = time.perf_counter()
        list(ex.map(_oracle_colouring, [g_spec] * colourings, [k] * colourings, [e] * colourings,
                    [root] * colourings, [1] * colourings, range(colourings)))
        wall = time.perf_counter() - t
    return U_per_colouring * colourings / wall, wall


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    s, dt, desc, g, k, e, root = oracle_sample(wl, target_s=args.ref_seconds / 4)
    U = plan_updates_host(g, k, e, root)
    cores = host_cores()
    spec = wl["graph"] if s is None else ("rmat", s, wl["graph"][2])
    # each step: one colouring per host core, in parallel (a bounded sample)
    steps = []
    for i in range(args.steps):
        rate, wall = oracle_cores_rate(spec, k, e, root, U, cores, cores)
        steps.append(wall)
    tot = sum(steps)
    value = U * cores * len(steps) / tot
    desc += f"; one colouring per core on {cores} cores per step"
    line = {"impl": "reference", "metric": "edge_colourset_updates_per_s", "value": value,
            "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u256", "data": "synthetic",
            "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle", "sample": desc},
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


def fifo_latencies(arrivals, service):
    """Arrival-to-result latencies of one server taking requests in arrival
    order: request i starts when it has arrived and request i - 1 is done."""
    done, out = 0.0, []
    for a, sv in zip(arrivals, service):
        done = max(done, a) + sv
        out.append(done - a)
    return out


def pctl(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * (len(xs) - 1) + 0.5))] if xs else None


def run_serving(args):
    """Continuous-batching serving: resident R-MAT graphs (scales 16..max) plus
    an Erdos-Renyi graph (n = 2^20, degree 16); requests with Poisson arrivals,
    each a uniform labelled tree (Pruefer sequence) with k in 5..12 and 1..16
    colourings.  The served run submits every request at its arrival time and
    reports p50/p99 latency (arrival to result) and throughput.  The same
    requests are also run one after another, on the same GPU, in two plain
    forms: through cc_count (each request's colourings batched into passes) and
    with one colouring per pass; their latencies under the same arrivals are
    those of a single FIFO server with the measured service times.  A second,
    lighter arrival rate (a sustainable load) is served as well.  Every served
    result must equal the plain results."""
    import torch

    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    rng = np.random.default_rng(2024)
    scales = list(range(16, args.serve_max_scale + 1))
    graphs = [gg.rmat_graph(sc, seed=sc) for sc in scales] + [gg.er_graph(1 << 20, 16, seed=7)]
    budget = min(int(args.budget_gb * (1 << 30)) if args.budget_gb else 250 << 30,
                 int(torch.cuda.mem_get_info(0)[0] * 0.9))

    def make_requests(n, rate, seed0):
        r_rng = np.random.default_rng(seed0)
        out, t = [], 0.0
        for i in range(n):
            t += r_rng.exponential(1.0 / rate)
            k = int(r_rng.integers(5, 13))
            out.append(dict(at=t, g=int(r_rng.integers(0, len(graphs))), k=k, e=gg.prufer_tree(k, seed0 * 100_000 + i),
                            n_iter=int(r_rng.integers(1, 17)), seed=int(r_rng.integers(0, 2 ** 40))))
        return out

    def served(ctx, gids, reqs):
        for r in reqs:
            r["tid"] = ctx.template_load(r["k"], r["e"])
        torch.cuda.synchronize()
        start = time.perf_counter()
        ids = []
        for r in reqs:
            now = time.perf_counter() - start
            if r["at"] > now:
                time.sleep(r["at"] - now)
            ids.append((ctx.submit(gids[r["g"]], r["tid"], r["seed"], r["n_iter"]), r))
        for rid, r in ids:
            try:
                r["served"] = ctx.wait(rid, r["n_iter"], timeout_s=7200)["counts"]
            except cc.CCError as e:
                r["served"] = e.status
        return time.perf_counter() - start, ctx.serve_stats()

    def plain(ctx, gids, reqs, key):
        # one request after another; the service time of each, and its result
        for r in reqs:
            tid = ctx.template_load(r["k"], r["e"])
            torch.cuda.synchronize()
            t = time.perf_counter()
            try:
                r[key] = ctx.count(gids[r["g"]], tid, seed=r["seed"], n_iter=r["n_iter"])["counts"]
            except cc.CCError as e:
                r[key] = e.status
            r[key + "_s"] = time.perf_counter() - t
            ctx.template_free(tid)

    reqs = make_requests(args.requests, args.rate, 2024)
    for r in reqs:
        r["U"] = plan_updates_host(graphs[r["g"]], r["k"], r["e"], 0) * r["n_iter"]
    # served at the offered rate
    ctx = cc.Context(budget_bytes=budget, max_slots=args.serve_slots, batch=0, autotune=0)
    gids = [ctx.graph_load(g) for g in graphs]
    with ClockSampler(0) as clk:
        served_s, st = served(ctx, gids, reqs)
    # the same requests, one after another: batched passes, then one colouring per pass
    plain(ctx, gids, reqs, "plain")
    ctx.close()
    ctx1 = cc.Context(budget_bytes=budget, batch=1, autotune=0)
    gids1 = [ctx1.graph_load(g) for g in graphs]
    plain(ctx1, gids1, reqs, "one")
    ctx1.close()
    ok = [r for r in reqs if not isinstance(r["plain"], int)]
    U = sum(r["U"] for r in ok)
    arrivals = [r["at"] for r in reqs]

    def plain_summary(key):
        lat = fifo_latencies(arrivals, [r[key + "_s"] for r in reqs])
        busy = sum(r[key + "_s"] for r in reqs)
        return {"busy_s": busy, "requests_per_s_busy": len(reqs) / busy, "updates_per_s_busy": U / busy,
                "p50_latency_s": pctl(lat, 0.5), "p99_latency_s": pctl(lat, 0.99),
                "makespan_s": max(a + l for a, l in zip(arrivals, lat))}

    differ = sum(r["served"] != r["plain"] for r in reqs) + sum(r["one"] != r["plain"] for r in ok)

    def brief(x):
        return x if isinstance(x, int) else [len(x), x[0] if x else None]

    mismatches = [{"i": i, "graph": graphs[r["g"]].name, "k": r["k"], "n_iter": r["n_iter"],
                   "served": brief(r["served"]), "plain": brief(r["plain"]), "one": brief(r["one"]),
                   "first_differing": next((j for j, (a, b) in enumerate(zip(r["served"], r["plain"])) if a != b), None)
                   if not isinstance(r["served"], int) and not isinstance(r["plain"], int) else None}
                  for i, r in enumerate(reqs) if r["served"] != r["plain"] or r["one"] != r["plain"]][:12]
    # a sustainable load: fewer, sparser requests, served only (the plain forms'
    # service times do not depend on the rate)
    light = make_requests(args.light_requests, args.light_rate, 4048)
    ctx = cc.Context(budget_bytes=budget, max_slots=args.serve_slots, batch=0, autotune=0)
    gids = [ctx.graph_load(g) for g in graphs]
    light_s, st_l = served(ctx, gids, light)
    plain(ctx, gids, light, "plain")
    ctx.close()
    light_ok = [r for r in light if not isinstance(r["plain"], int)]
    differ += sum(r["served"] != r["plain"] for r in light)
    lat_l = fifo_latencies([r["at"] for r in light], [r["plain_s"] for r in light])
    line = {"metric": "served_p99_latency_s", "value": st["p99_latency_s"], "unit": "s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": served_s * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64..u256", "data": "synthetic",
            "config": {"workload": "serve", "graphs": [g.name for g in graphs], "requests": args.requests,
                       "rate_per_s": args.rate, "slots": args.serve_slots,
                       "batch": "up to 16 colourings per pass, fewer when the budget requires", "k": "5..12",
                       "colourings": "1..16", "arrival_span_s": arrivals[-1]},
            "serving": {"p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
                        "mean_latency_s": st["mean_latency_s"], "completed": st["completed"],
                        "requests_per_s": st["completed"] / served_s, "updates_per_s": U / served_s,
                        "busy_s": st["busy_seconds"], "admissions_deferred": st["admissions_deferred"],
                        "passes": st["passes"], "shared_passes": st["shared_passes"],
                        "colourings_run": st["colourings_run"],
                        "refused_over_budget": len(reqs) - len(ok), "results_differ_from_plain": differ,
                        "mismatches": mismatches},
            "plain_sequential": plain_summary("plain"),
            "one_colouring_per_launch": plain_summary("one"),
            "sustainable": {"requests": len(light), "rate_per_s": args.light_rate,
                            "served_p50_latency_s": st_l["p50_latency_s"], "served_p99_latency_s": st_l["p99_latency_s"],
                            "served_requests_per_s": st_l["completed"] / light_s,
                            "shared_passes": st_l["shared_passes"], "passes": st_l["passes"],
                            "plain_sequential_p50_latency_s": pctl(lat_l, 0.5),
                            "plain_sequential_p99_latency_s": pctl(lat_l, 0.99),
                            "refused_over_budget": len(light) - len(light_ok)},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_multi(args):
    """Graphlet-frequency counting: every tree on k = 7 vertices (11 templates)
    on R-MAT scale 20 over the same colourings, as one merged count
    (cc_count_multi: shared rooted sub-templates, one colouring and histogram
    per pass) and as one count per template.  Results must be identical."""
    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    g = make_graph(("rmat", 20, 20))
    trees = gg.all_trees(7)
    n_iter = args.n_iter or 16
    ctx = cc.Context(budget_bytes=int((args.budget_gb or 60) * (1 << 30)), batch=16)
    gid = ctx.graph_load(g)
    tids = [ctx.template_load(7, e) for e in trees]
    info = ctx.multi_plan_info(gid, tids, n_iter)
    for _ in range(max(1, args.warmup)):
        ctx.count_multi(gid, tids, seed=1, n_iter=n_iter)
        for t in tids:
            ctx.count(gid, t, seed=1, n_iter=n_iter)
    merged_s = separate_s = 0.0
    differ = 0
    for step in range(args.steps):
        seed = 100 + step
        res = ctx.count_multi(gid, tids, seed=seed, n_iter=n_iter)
        merged_s += res[0]["device_seconds"]
        for t, m in zip(tids, res):
            alone = ctx.count(gid, t, seed=seed, n_iter=n_iter)
            separate_s += alone["device_seconds"]
            differ += alone["counts"] != m["counts"]
    per_step = n_iter * len(tids)
    line = {"metric": "template_colourings_per_s", "value": per_step * args.steps / merged_s,
            "unit": "template-colourings/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": merged_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64..u128", "data": "synthetic",
            "config": {"workload": "rmat20_trees7", "graph": g.name, "n": g.n, "templates": len(tids),
                       "colourings_per_step": n_iter},
            "multi": {"merged_s_per_step": merged_s / args.steps, "separate_s_per_step": separate_s / args.steps,
                      "speedup": separate_s / merged_s, "tables_merged": info["chains"],
                      "tables_separate": info["chains_separate"],
                      "updates_per_colouring_merged": info["updates_per_colouring"],
                      "updates_per_colouring_separate": info["updates_per_colouring_separate"],
                      "results_differ": differ}}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_graph_batch(args):
    """Many small graphs in one launch: N Erdos-Renyi graphs of the tiny
    workload's shape (n = 2000, average degree 8, each its own seed) with the
    5-vertex path, one colouring each, counted as one resident batch
    (cc_graph_load_batch + cc_count_batch: every DP launch covers all N) and
    as N separate counts of the same graphs (one graph per launch).  Per-graph
    counts must be identical."""
    import torch

    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    n_graphs = args.graphs
    gs = [gg.er_graph(2000, 8, seed=1000 + i) for i in range(n_graphs)]
    k, e = gg.template_edges("P5")
    n_iter = args.n_iter or 1
    ctx = cc.Context(budget_bytes=8 << 30, batch=16, timing=0)
    bid = ctx.graph_load_batch(gs)
    gids = [ctx.graph_load(g) for g in gs]
    tid = ctx.template_load(k, e, 2)
    U = sum(plan_updates_host(g, k, e, 2) for g in gs) * n_iter
    for i in range(args.warmup):
        ctx.count_batch(bid, tid, seed=77, n_iter=n_iter, first_iter=i * n_iter)
        for gi in gids:
            ctx.count(gi, tid, seed=77, n_iter=n_iter, first_iter=i * n_iter)
    bat_dev = bat_wall = sep_dev = sep_wall = 0.0
    bat_l = sep_l = 0
    differ = 0
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = ctx.count_batch(bid, tid, seed=4321, n_iter=n_iter, first_iter=i * n_iter)
            bat_wall += time.perf_counter() - t
            bat_dev += r["device_seconds"]
            bat_l += r["kernel_launches"]
            t = time.perf_counter()
            for gi, gid in enumerate(gids):
                a = ctx.count(gid, tid, seed=4321, n_iter=n_iter, first_iter=i * n_iter)
                sep_dev += a["device_seconds"]
                sep_l += a["kernel_launches"]
                differ += a["counts"] != r["counts"][gi]
            sep_wall += time.perf_counter() - t
    per = n_graphs * args.steps
    line = {"metric": "edge_colourset_updates_per_s", "value": U * args.steps / bat_dev, "unit": "updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * bat_dev / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "er2000_p5_batch", "graphs_per_launch": n_graphs, "n_per_graph": 2000,
                       "avg_degree": 8, "template": "P5", "colourings_per_graph": n_iter,
                       "l2": "inputs smaller than L2 (launch-bound workload)"},
            "graph_batch": {"batched_us_per_graph": 1e6 * bat_dev / per, "separate_us_per_graph": 1e6 * sep_dev / per,
                            "batched_wall_us_per_graph": 1e6 * bat_wall / per,
                            "separate_wall_us_per_graph": 1e6 * sep_wall / per,
                            "speedup_device": sep_dev / bat_dev, "speedup_wall": sep_wall / bat_wall,
                            "launches_batched_per_step": bat_l / args.steps,
                            "launches_separate_per_step": sep_l / args.steps, "results_differ": differ},
            "gpu_launches": int(bat_l), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_compare_plain(args):
    """The batched form against the plain one-colouring-per-launch form on the
    same GPU, graph, template and colourings (the default workload here is
    R-MAT scale 20 / caterpillar-10, 64 colourings).  Plain: one colouring per
    pass, gather and combine as separate launches for every DP stage, no CUDA
    graph, no autotuning.  Batched: as many colourings per pass as the budget
    holds (at most 16), fused gather + combine kernels, every pass replayed
    from a captured CUDA graph, and the shape (split threshold, column
    segments, vertex-block size) chosen by the autotuner on the first count.
    The counts of the two forms must be identical."""
    import torch

    from paper_1804_09764_gb300 import build as B
    from paper_1804_09764_gb300 import cc

    B.build()
    wl = dict(WORKLOADS[args.workload])
    n_iter = args.n_iter or wl["n_iter"]
    g = make_graph(wl["graph"])
    k, e = gg.template_edges(wl["template"])
    budget = int(args.budget_gb * (1 << 30)) if args.budget_gb else wl["budget"]
    budget = min(budget, int(torch.cuda.mem_get_info(0)[0] * 0.9))
    forms = {"plain": dict(batch=1, fused=0, use_cuda_graph=0, autotune=0),
             "batched": dict(batch=0, fused=1, use_cuda_graph=1, autotune=1)}
    out, counts = {}, {}
    for name, opt in forms.items():
        # no per-kernel timing (it keeps passes out of CUDA graphs): device time
        # is the CUDA-event span of each count's passes on the context's stream
        ctx = cc.Context(budget_bytes=budget, timing=0, **opt)
        gid = ctx.graph_load(g)
        tid = ctx.template_load(k, e, wl["root"])
        for i in range(args.warmup):  # the batched form tunes and captures here
            ctx.count(gid, tid, seed=4242, n_iter=n_iter, first_iter=i * n_iter)
        dev = wall = 0.0
        launches = 0
        got = []
        with ClockSampler(0) as clk:
            for i in range(args.steps):
                torch.cuda.synchronize()
                t = time.perf_counter()
                r = ctx.count(gid, tid, seed=12345, n_iter=n_iter, first_iter=i * n_iter)
                wall += time.perf_counter() - t
                dev += r["device_seconds"]
                launches += r["kernel_launches"]
                got.append(r["counts"])
        info = ctx.plan_info(gid, tid)
        U = info["updates_per_colouring"] * n_iter * args.steps
        out[name] = {"value": U / dev, "ms_per_step": 1e3 * dev / args.steps,
                     "wall_ms_per_step": 1e3 * wall / args.steps, "gpu_launches_per_step": launches / args.steps,
                     "options": opt, "batch": info["batch"], "passes_per_step": -(-n_iter // info["batch"]),
                     "split_threshold": info["split_threshold"], "col_chunks": info.get("col_chunks"),
                     "blocks": info["n_blocks"], "block_vertices": info["block_vertices"],
                     "workspace_gb": info["workspace_bytes"] / 1e9,
                     "clocks": clk.summary()}
        counts[name] = got
        ctx.close()
    pl, bt = out["plain"], out["batched"]
    line = {"metric": "edge_colourset_updates_per_s", "value": bt["value"], "unit": "updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": bt["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64..u128",
            "data": "synthetic",
            "config": {"workload": args.workload, "graph": g.name, "n": g.n, "m": g.m, "template": wl["template"],
                       "k": k, "colourings_per_step": n_iter, "l2": "inputs larger than L2"},
            "compare_plain": {"plain": pl, "batched": bt, "speedup": bt["value"] / pl["value"],
                              "identical_counts": counts["plain"] == counts["batched"]},
            "gpu_launches": int(bt["gpu_launches_per_step"] * args.steps), "clocks": bt["clocks"]}
    print(json.dumps(line), flush=True)


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
    ap.add_argument("--gather-mode", type=int, default=1,
                    help="1 persistent warp gather, 4 rows in flight (default); 6: 2 rows in flight; 5 one-pass warp "
                         "gather; 0 bulk-copy (TMA) ring; 2 warp 16-byte vectors; 3 group; 4 as 6 + L2 prefetch")
    ap.add_argument("--budget-gb", type=float, default=0, help="HBM arena size (0: the workload's)")
    ap.add_argument("--fused", type=int, default=1, help="1: fused gather + a=1 combine kernel")
    ap.add_argument("--autotune", type=int, default=0, help="1: time every gather variant per site on the first pass")
    ap.add_argument("--vertex-order", type=int, default=0, help="0: by decreasing degree, 1: input order")
    ap.add_argument("--multi", action="store_true",
                    help="graphlet-frequency run: all 11 trees on 7 vertices, merged vs one count each")
    ap.add_argument("--l2-persist-mb", type=int, default=0,
                    help="MiB of L2 kept for the hub rows of each gathered table (0: none)")
    ap.add_argument("--col-chunks", type=int, default=0,
                    help="column segments per neighbour row in the persistent gathers (0: one warp sweep each, "
                         "whole rows in the fused kernels; 1: whole rows)")
    ap.add_argument("--serve", action="store_true", help="run the serving scenario instead")
    ap.add_argument("--graph-batch", action="store_true",
                    help="many small graphs in one launch against one graph per count")
    ap.add_argument("--graphs", type=int, default=1000, help="graphs of the --graph-batch run")
    ap.add_argument("--compare-plain", action="store_true",
                    help="batched + CUDA graph + autotuned form against one colouring per pass, unfused, no graph")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--light-requests", type=int, default=300, help="requests of the sustainable-rate serving run")
    ap.add_argument("--light-rate", type=float, default=4.0, help="arrival rate of the sustainable-rate serving run")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-max-scale", type=int, default=22)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--full-rows", type=int, default=0,
                    help="1: gathers read whole neighbour rows (0: skip the entries zero by Eq. 1 at batch 1)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.n_iter:
        wl["n_iter"] = args.n_iter
    rank, world, local = dist_env()

    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if args.serve:
        if rank == 0:
            run_serving(args)
        return
    if args.multi:
        if rank == 0:
            run_multi(args)
        return
    if args.graph_batch:
        if rank == 0:
            run_graph_batch(args)
        return
    if args.compare_plain:
        if args.workload == DEFAULT:
            args.workload = "rmat20_caterpillar10"
        if rank == 0:
            run_compare_plain(args)
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
    budget = int(args.budget_gb * (1 << 30)) if args.budget_gb else wl["budget"]
    budget = min(budget, int(torch.cuda.mem_get_info(local)[0] * 0.9))
    ctx = cc.Context(device=local, budget_bytes=budget, timing=1, split_threshold=args.split, batch=args.batch,
                     block_vertices=args.block, gather_mode=args.gather_mode, fused=args.fused,
                     autotune=args.autotune, vertex_order=args.vertex_order, col_chunks=args.col_chunks,
                     l2_persist_mb=args.l2_persist_mb, full_rows=args.full_rows)
    gid = ctx.graph_load(g)
    tlab = glab = None
    if wl.get("labels"):
        rng = np.random.default_rng(1234)
        glab = rng.integers(0, wl["labels"], g.n, dtype=np.uint8)
        ctx.graph_set_labels(gid, glab)
        tlab = rng.integers(0, wl["labels"], k, dtype=np.uint8)
    tid = ctx.template_load(k, e, wl["root"], labels=tlab)
    n_iter = wl["n_iter"]

    def step(i):
        return ctx.count(gid, tid, seed=12345, n_iter=n_iter, first_iter=replica_first_iter(rank, world, i, n_iter))

    for i in range(args.warmup):
        step(i)
    ctx.kernel_stats_reset()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    dev_s = 0.0
    launches = 0
    mine = []  # (colouring index, count) of the timed steps
    with ClockSampler(local) as clk:
        t_start = time.perf_counter()
        for i in range(args.steps):
            r = step(args.warmup + i)
            dev_s += r["device_seconds"]
            launches += r["kernel_launches"]
            j0 = replica_first_iter(rank, world, args.warmup + i, n_iter)
            mine.extend((j0 + b, c) for b, c in enumerate(r["counts"]))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - t_start
    ks = ctx.kernel_stats()
    insts = ctx.kernel_instances()  # the timed steps only (before the end-to-end counts)
    info = ctx.plan_info(gid, tid)  # the plan the timed counts used
    elapsed = dev_s
    rcheck = None
    if world > 1:
        elapsed = max_over_ranks(elapsed, device=f"cuda:{local}")
        per_rank = [None] * world
        torch.distributed.all_gather_object(per_rank, mine)
        if rank == 0:
            rcheck = replica_check(per_rank, lambda j: ctx.count(gid, tid, seed=12345, n_iter=1,
                                                                 first_iter=j)["counts"][0])
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
            if glab is not None:
                ctx.graph_set_labels(gid2, glab)
            r = ctx.count(gid2, tid, seed=777, n_iter=n_iter, first_iter=replica_first_iter(rank, world, i, n_iter))
            ctx.graph_free(gid2)
            ctx2_t.append(time.perf_counter() - t)
        et = sum(ctx2_t[1:])
        if world > 1:
            et = max_over_ranks(et, device=f"cuda:{local}")
        e2e = {"value": info["updates_per_colouring"] * n_iter * args.steps * world / et, "unit": "updates/s",
               "h2d_bytes_per_step": int(rp.numel() * 8 + ci.numel() * 4 + (0 if glab is None else glab.size)),
               "d2h_bytes_per_step": int(n_iter * 4 * 8)}

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return
    peak, peak_kind = measured_peaks()
    kinds = {k_: v for k_, v in ks.items() if isinstance(v, dict) and v["launches"] > 0}
    # the dominant kernel: the instantiation with the most timed device time
    timed = [(kind, nm, st) for kind, d in insts.items() for nm, st in d.items() if st["seconds"] > 0]
    dkind, dname, d = max(timed, key=lambda x: x[2]["seconds"])
    kernel_s = sum(v["seconds"] for v in kinds.values())
    achieved = d["bytes"] / d["seconds"] / 1e9
    avg_s = d["seconds"] / d["timed_launches"]
    traffic = profiled_traffic(dname, args.workload)
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": traffic,
                "dram_achieved": traffic / avg_s / 1e9 if traffic else None,
                "dram_frac": traffic / avg_s / 1e9 / peak if traffic else None,
                "algorithmic_bytes_per_launch": d["bytes"] / d["timed_launches"],
                "launches": d["timed_launches"], "avg_launch_ms": 1e3 * avg_s,
                "share_of_kernel_time": d["seconds"] / kernel_s}
    if dkind == "combine" and info["limb_products_per_colouring"] > 0:
        d = kinds["combine"]
        # the general combine is bound by its wide multiply-adds: 64-bit limb
        # products per second against the rate the GPU sustains on registers
        lp = info["limb_products_per_colouring"] * n_iter * args.steps
        alu_peak = ctx.limb_product_rate()
        a_alu = lp / d["seconds"] / 1e12
        roofline.update({"bound": "alu", "kernel": "combine (all instantiations)", "achieved": a_alu,
                         "peak": alu_peak / 1e12,
                         "unit": "T limb-products/s", "frac": a_alu / (alu_peak / 1e12),
                         "peak_kind": "measured (cc_limb_product_rate: register-resident 64-bit multiply-adds)",
                         "hbm_achieved_gbs": d["bytes"] / d["seconds"] / 1e9, "hbm_peak_gbs": peak,
                         "limb_products_per_launch": lp / d["launches"], "launches": d["launches"],
                         "avg_launch_ms": 1e3 * d["seconds"] / d["launches"],
                         "share_of_kernel_time": d["seconds"] / kernel_s, "traffic": None,
                         "dram_achieved": None, "dram_frac": None})
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        # a bounded sample: the oracle on an R-MAT graph of the workload's
        # parameters whose one colouring takes a few seconds, one colouring per
        # host core in parallel
        s, dt, desc, gs, k2, e2, root2 = oracle_sample(wl, target_s=12.0)
        Us = plan_updates_host(gs, k2, e2, root2)
        cores = host_cores()
        spec = wl["graph"] if s is None else ("rmat", s, wl["graph"][2])
        rate, wall = oracle_cores_rate(spec, k2, e2, root2, Us, cores, cores)
        cpu = {"value": rate, "unit": "updates/s", "cores": cores, "kind": "oracle",
               "sample": desc + f"; {cores} colourings, one per core, in {wall:.1f} s",
               "single_core": {"value": Us / dt, "seconds": round(dt, 2)}}
    line = {
        "metric": "edge_colourset_updates_per_s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64" if info["limbs_root"] == 1 else f"u64..u{64 * info['limbs_root']}",
        "data": "synthetic",
        "config": {"workload": args.workload, "graph": g.name, "n": g.n, "m": g.m, "n_active": info["n_active"],
                   "template": wl["template"], "k": k, "root": info["root"], "colourings_per_step": n_iter,
                   "labels": wl.get("labels", 0),
                   "batch": info["batch"], "blocks": info["n_blocks"], "limbs_root": info["limbs_root"],
                   "workspace_gb": info["workspace_bytes"] / 1e9,
                   # the same plan's device memory without freeing tables early, without
                   # vertex blocks, and with neither (no memory is allocated for these)
                   "workspace_no_reuse_gb": info["workspace_no_reuse_bytes"] / 1e9,
                   "workspace_no_blocks_gb": info["workspace_no_blocks_bytes"] / 1e9,
                   "workspace_naive_gb": info["workspace_naive_bytes"] / 1e9,
                   "l2": "inputs larger than L2",
                   "updates_per_colouring": info["updates_per_colouring"],
                   "algorithmic_bytes_per_colouring": info["algorithmic_bytes_per_colouring"],
                   "graph_gen_s": round(gen_s, 1), "wall_s": round(wall, 3), "fused": bool(args.fused), "autotune": bool(args.autotune),
                   "vertex_order": "degree" if args.vertex_order == 0 else "input",
                   "col_chunks": args.col_chunks or "auto", "l2_persist_mb": args.l2_persist_mb,
                   # entries of a neighbour's row whose set lacks its colour (zero by Eq. 1):
                   # skipped by the gathers in one-colouring passes, or read with the row
                   "absent_entries": "skipped" if any("neighbour_colours_kernel" in v for v in insts.values())
                   else "read",
                   "gather": {0: "bulk-copy (TMA)", 1: "persistent warp per row, 4 rows in flight",
                              2: "warp (16-byte vectors)", 3: "group (row per 32-256 threads)",
                              4: "persistent warp + L2 prefetch", 5: "warp per row, one pass",
                              6: "persistent warp per row, 2 rows in flight"}[args.gather_mode]},
        "hbm_frac_step": info["algorithmic_bytes_per_colouring"] * n_iter * args.steps / elapsed / 1e9 / peak,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "replica_check": rcheck,
        "clocks": clk.summary(),
        "kernels": {k_: {"launches": v["launches"], "ms": round(1e3 * v["seconds"], 3),
                         "GBps": (v["bytes"] / v["seconds"] / 1e9) if v["seconds"] else None,
                         "instances": {nm: {"launches": st["launches"], "ms": round(1e3 * st["seconds"], 3),
                                            "GBps": (st["bytes"] / st["seconds"] / 1e9) if st["seconds"] else None}
                                       for nm, st in insts[k_].items()}}
                    for k_, v in kinds.items()},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.barrier()


if __name__ == "__main__":
    main()
