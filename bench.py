"""Benchmark: full multilevel LP partition on the GPU, reported as LP GTEPS.

A step is one complete partition (coarsening LP + contraction per level, initial partitioning,
projection + LP refinement per level, degree-0 placement, evaluation) of one synthetic graph whose CSR
is resident in HBM when the timed region starts. value = LP edges traversed per step (CSR entries
scanned by all LP sub-rounds of the partition, counted by the library) / device time per step.

Default workload: the largest configuration, R-MAT scale 26 (67M vertices, about 2.1G CSR entries),
edge factor 16, integer edge weights in [1,8], k=64, eps=0.03, seed 1. Other workloads: rgg20 (random
geometric graph 2^20), grid256, rmat24, batch512.

The line carries, besides value: the LP kernel's HBM roofline (all LP launches, and the level-0
coarsening launch alone), LP-only GTEPS (LP edges over LP kernel time), an end-to-end number through
gp_partition_host from pinned host buffers, the CPU oracle timed on all host cores on a bounded sample
of the workload, a check of the GPU result against the oracle's stored digests of the full-size
workload, and comparisons at the same seed: the learned edge scorer against plain LP, and the batch of
512 uneven graphs in one call against a per-graph loop.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
                       [--mode plain|learned] [--no-compare] [--learned-seeds S]
--workload batch512 makes the batched call itself the timed step (value: LP GTEPS of the batch).
For N > 1 the script runs under torch.distributed.run; every rank partitions its own replica
(replicas only: the single-graph path does not shard), so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "rgg20": dict(kind="rgg", n=1 << 20, deg=12.0, k=16, desc="random geometric graph 2^20 vertices, avg degree 12, unit weights, k=16, eps=0.03, seed 1"),
    "grid256": dict(kind="grid", a=256, b=256, k=2, desc="2D 4-neighbour grid 256x256, unit weights, k=2, eps=0.03, seed 1"),
    "rmat24": dict(kind="rmat", scale=24, ef=16, k=16, weighted=False, desc="R-MAT scale 24, edge factor 16, (0.57,0.19,0.19), symmetrised, unit weights, k=16, eps=0.03, seed 1"),
    "rmat26w": dict(kind="rmat", scale=26, ef=16, k=64, weighted=True, desc="R-MAT scale 26, edge factor 16, edge weights in [1,8], k=64, eps=0.03, seed 1"),
    # a 1/16-size stand-in of rmat26w for profiler captures
    "rmat22w": dict(kind="rmat", scale=22, ef=16, k=64, weighted=True, desc="R-MAT scale 22, edge factor 16, edge weights in [1,8], k=64, eps=0.03, seed 1"),
    "batch512": dict(kind="batch", count=512, desc="batch of 512 uneven graphs (grids and RGGs, 1k-200k vertices, log-uniform), unit weights, k in {2,4,8}, eps=0.03, seed 1"),
}
EPS, SEED = 0.03, 1
METRIC = "LP GTEPS + ms/partition at equal cut (plain vs learned/batched), % HBM peak"


def make_batch(count: int = 512):
    import graphgen as gg
    specs = gg.batch_specs(count, seed=SEED)
    return specs, [gg.batch_graph(sp) for sp in specs]


def family_graphs(name: str):
    """Training graphs for the learned scorer: the workload's family at a smaller size, other seeds."""
    import graphgen as gg
    w = WORKLOADS[name]
    if w["kind"] == "rgg":
        return [gg.rgg(1 << 16, w["deg"], s) for s in (101, 102)]
    if w["kind"] == "grid":
        return [gg.grid(128, 128), gg.grid(96, 160)]
    return [gg.rmat(16, w["ef"], seed=s, weighted=w["weighted"]) for s in (101, 102)]


def train_scorer(gp, name: str, k: int):
    """Trains the 8-32-1 scorer on which edges plain partitions of same-family graphs leave uncut. The
    classes are balanced first (every cut edge and as many uncut edges, taken by a seeded draw): on mesh
    graphs more than 99% of the edges are uncut, and a scorer trained on them all learns a constant."""
    import torch
    feats, ys = [], []
    rng = np.random.default_rng(SEED)
    for g in family_graphs(name):
        dg = gp.DeviceGraph.from_host(g)
        part, _ = gp.partition(dg, k, EPS, SEED)
        p = part.cpu().numpy()
        src = np.repeat(np.arange(g.n), np.diff(g.off))
        y = p[src] == p[g.adj]
        pos, neg = np.flatnonzero(y), np.flatnonzero(~y)
        keep = np.sort(np.concatenate([neg, rng.choice(pos, min(len(pos), len(neg)), replace=False)]))
        idx = torch.from_numpy(keep).cuda()
        feats.append(gp.edge_features(dg, 0)[idx].contiguous())
        ys.append(torch.from_numpy(y[keep].astype(np.float32)).cuda())
    rng = np.random.default_rng(SEED)
    mlp = gp.mlp_pack(rng.normal(0, 0.2, (32, 8)), rng.normal(0, 0.1, 32), rng.normal(0, 0.2, 32),
                      float(rng.normal(0, 0.1)))
    losses = gp.mlp_train(torch.cat(feats), torch.cat(ys), mlp, 300, 1e-2)
    return mlp, [float(losses[0]), float(losses[-1])]


def time_steps(fn, steps, flush):
    """Device time (ms) of `steps` calls of fn, events on the current stream, L2 flushed between."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    out = None
    for i in range(steps):
        flush.fill_(i)
        ev[i][0].record(stream)
        out = fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev), out


def compare_learned(gp, name, g, dg, k, steps, flush, plain_ms, plain_res, nseeds=10):
    """Learned against plain LP on the same graph at seeds 1..nseeds (geometric means of the per-seed cut
    and time ratios), plus the timed learned run at the bench's own seed."""
    import math
    mlp, loss = train_scorer(gp, name, k)
    params = gp.default_params(mode=gp.MODE_LEARNED)
    params.mlp = mlp.data_ptr()
    if plain_ms > 2000:  # long partitions: one timed learned run, no warm-up
        steps = 1
    else:
        gp.partition(dg, k, EPS, SEED, params)
    ms, (_, res) = time_steps(lambda: gp.partition(dg, k, EPS, SEED, params), steps, flush)
    per_seed = []
    for sd in range(1, nseeds + 1):
        if sd == SEED and plain_ms > 2000:  # the bench's own seed: the runs above
            pm, rp, lm, rl = plain_ms, plain_res, ms / steps, res
        else:
            pm, (_, rp) = time_steps(lambda: gp.partition(dg, k, EPS, sd), 1, flush)
            lm, (_, rl) = time_steps(lambda: gp.partition(dg, k, EPS, sd, params), 1, flush)
        per_seed.append({"seed": sd, "plain_cut": rp.cut, "learned_cut": rl.cut, "plain_ms": pm, "learned_ms": lm,
                         "learned_imbalanced": rl.imbalanced})
    gm = lambda xs: math.exp(sum(math.log(x) for x in xs) / len(xs))
    return {"ms_per_partition": ms / steps, "gteps": res.lp_edges * steps / (ms * 1e-3) / 1e9, "cut": res.cut,
            "imbalanced": res.imbalanced, "plain_cut": plain_res.cut, "plain_ms_per_partition": plain_ms,
            "cut_ratio_learned_over_plain": res.cut / max(plain_res.cut, 1),
            "time_ratio_learned_over_plain": (ms / steps) / plain_ms, "levels": res.levels,
            "seeds": {"count": nseeds, "geomean_cut_ratio": gm([x["learned_cut"] / max(x["plain_cut"], 1) for x in per_seed]),
                           "geomean_time_ratio": gm([x["learned_ms"] / x["plain_ms"] for x in per_seed]),
                           "learned_better_or_equal": sum(x["learned_cut"] <= x["plain_cut"] for x in per_seed),
                           "per_seed": per_seed},
            "training": {"graphs": "2 same-family graphs, seeds 101-102", "steps": 300, "lr": 1e-2,
                         "target": "edge left uncut by the plain partition, classes balanced",
                         "bce_first_last": loss},
            "note": "learned is reported as measured; worse cuts are not hidden"}


def compare_ip_tries(gp, name, dg, k, ms_step, flush):
    """Cut and time against the number of initial-partitioning tries I (Section IV-B runs the tries in
    parallel; a larger I gave a lower cut in the paper's Section VI). On workloads whose partition
    takes more than 2 s the sweep runs on the random geometric graph 2^20, k=16 instead."""
    import graphgen as gg
    if ms_step > 2000:
        name, k = "rgg20", 16
        dg = gp.DeviceGraph.from_host(gg.rgg(1 << 20, 12.0, SEED))
    out = {"graph": WORKLOADS[name]["desc"], "per_tries": []}
    for tries in (1, 2, 4, 8, 16):
        params = gp.default_params(ip_tries=tries)
        gp.partition(dg, k, EPS, SEED, params)
        ms, (_, r) = time_steps(lambda: gp.partition(dg, k, EPS, SEED, params), 3, flush)
        out["per_tries"].append({"ip_tries": tries, "cut": r.cut, "best_try": r.best_try, "imbalanced": r.imbalanced,
                                 "ms_per_partition": ms / 3, "ms_initial": r.ms_initial})
    return out


def _side_graph(gp, name, dg, k, ms_step):
    """The workload itself, or the random geometric graph 2^20 (k=16) when a partition of the workload
    takes more than 2 s (the comparisons below run several partitions each)."""
    import graphgen as gg
    if ms_step > 2000 or WORKLOADS[name]["kind"] not in ("rgg", "grid"):
        return "rgg20", gp.DeviceGraph.from_host(gg.rgg(1 << 20, 12.0, SEED)), 16
    return name, dg, k


def compare_variants(gp, name, dg, k, ms_step, flush, seeds=10):
    """The §8(f) variants against the plain deterministic partition at seeds 1..seeds on a mesh graph:
    multi-try local search after every level (3 global iterations), matching coarsening, and the paper's
    asynchronous LP (non-deterministic: a comparator for what determinism costs). Geometric means of
    the per-seed cut and time ratios."""
    import math
    gname, g2, k2 = _side_graph(gp, name, dg, k, ms_step)
    variants = {"mls": dict(mls_global_iters=3), "matching": dict(coarsen=gp.COARSEN_MATCHING),
                "async_lp": dict(lp_async=1)}
    out = {"graph": WORKLOADS[gname]["desc"], "seeds": seeds}
    plain = []
    for sd in range(1, seeds + 1):
        ms, (_, r) = time_steps(lambda: gp.partition(g2, k2, EPS, sd), 1, flush)
        plain.append((r.cut, ms))
    gm = lambda xs: math.exp(sum(math.log(x) for x in xs) / len(xs))
    for vname, kw in variants.items():
        params = gp.default_params(**kw)
        gp.partition(g2, k2, EPS, 1, params)
        rows = []
        for sd in range(1, seeds + 1):
            ms, (_, r) = time_steps(lambda: gp.partition(g2, k2, EPS, sd, params), 1, flush)
            rows.append((r.cut, ms, r.imbalanced))
        out[vname] = {"geomean_cut_ratio": gm([a[0] / max(b[0], 1) for a, b in zip(rows, plain)]),
                      "geomean_time_ratio": gm([a[1] / b[1] for a, b in zip(rows, plain)]),
                      "better_or_equal": sum(a[0] <= b[0] for a, b in zip(rows, plain)),
                      "imbalanced": sum(a[2] for a in rows), "ms_per_partition": sum(a[1] for a in rows) / seeds,
                      "cuts": [a[0] for a in rows]}
    out["plain"] = {"cuts": [a for a, _ in plain], "ms_per_partition": sum(b for _, b in plain) / seeds}
    return out


def batch_items(gp, graphs):
    return [gp.DeviceGraph.from_host(g) for g in graphs]


def compare_batched(gp, steps, flush):
    specs, graphs = make_batch(512)
    dgs = batch_items(gp, graphs)
    ks = [sp.k for sp in specs]
    seeds = [sp.seed for sp in specs]
    big = max(range(len(graphs)), key=lambda i: graphs[i].n)
    dw, dc, _ = gp.autotune_schedule(dgs[big])
    params = gp.default_params(deg_warp=dw, deg_cta=dc)
    gp.partition_batch(dgs, ks, EPS, seeds, params)
    ms_b, (_, rb) = time_steps(lambda: gp.partition_batch(dgs, ks, EPS, seeds, params), steps, flush)
    loop_res = []

    def loop():
        loop_res.clear()
        for dg, k, sd in zip(dgs, ks, seeds):
            loop_res.append(gp.partition(dg, k, EPS, sd, params)[1])
        return loop_res

    loop()
    ms_l, _ = time_steps(loop, 1, flush)
    edges = sum(r.lp_edges for r in rb)
    return {"graphs": len(graphs), "n_total": int(sum(g.n for g in graphs)),
            "m_dir_total": int(sum(g.m_dir for g in graphs)), "schedule": {"deg_warp": dw, "deg_cta": dc},
            "batched_ms": ms_b / steps, "per_graph_loop_ms": ms_l, "speedup": ms_l / (ms_b / steps),
            "batched_gteps": edges * steps / (ms_b * 1e-3) / 1e9,
            "cuts_equal_to_loop": all(a.cut == b.cut for a, b in zip(rb, loop_res)),
            "total_cut": int(sum(r.cut for r in rb)), "imbalanced": int(sum(r.imbalanced for r in rb))}


def make_graph(name: str):
    import graphgen as gg
    w = WORKLOADS[name]
    if w["kind"] == "rgg":
        return gg.rgg(w["n"], w["deg"], SEED)
    if w["kind"] == "grid":
        return gg.grid(w["a"], w["b"])
    return gg.rmat(w["scale"], w["ef"], seed=SEED, weighted=w["weighted"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# committed ncu summaries giving DRAM bytes per k_lp launch (dram__bytes_read.sum + dram__bytes_write.sum),
# valid while the LP sources hash to the value recorded in them
TRAFFIC_SUMMARY = {"rmat26w": "profiles/k_lp_rmat_level0_dram.md"}
LP_SOURCES = ["paper_1710_08231_gb300/csrc/lp.cu", "paper_1710_08231_gb300/csrc/lp.cuh",
              "paper_1710_08231_gb300/csrc/gp_internal.cuh"]


def lp_traffic(workload: str, key: str):
    """DRAM bytes per k_lp launch (`key` = traffic_bytes_per_launch for the average over a partition's LP
    launches, level0_traffic_bytes_per_launch for the level-0 coarsening launch) from the committed ncu
    summary of this workload, or None when there is none or the LP sources changed since."""
    import hashlib
    path = os.path.join(ROOT, TRAFFIC_SUMMARY.get(workload, ""))
    if workload not in TRAFFIC_SUMMARY or not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            if ":" in line:
                k_, v_ = line.split(":", 1)
                fields[k_.strip().strip("`*- ")] = v_.strip().strip("`* ")
    h = hashlib.sha256()
    for src in LP_SOURCES:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    if fields.get("source_sha256") != h.hexdigest() or key not in fields:
        return None
    return float(fields[key])


def lp_roofline(prof, args, peak, peak_kind):
    """HBM roofline of k_lp from the library's per-launch CUDA events inside the timed region and its
    algorithmic byte counts: over every LP launch of the timed partitions, and over the level-0
    coarsening launches alone. Returns (roofline object, LP-only GTEPS)."""
    lp = [e for e in prof if e["name"].startswith("lp_persistent") and e["launches"] > 0 and e["ms"] > 0]
    if not lp:
        return None, None
    ms = sum(e["ms"] for e in lp)
    by = sum(e["bytes"] for e in lp)
    ed = sum(e["edges"] for e in lp)
    la = sum(e["launches"] for e in lp)
    achieved = by / (ms * 1e-3) / 1e9
    peak_src = "measured hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback 6.8 TB/s"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": lp_traffic(args.workload, "traffic_bytes_per_launch"),
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per k_lp launch, "
                              + TRAFFIC_SUMMARY.get(args.workload, "none"),
            "kernel": "k_lp (all LP launches of the timed partitions)", "launches": la,
            "ms_per_launch": ms / la, "bytes_per_launch": by / la, "peak_source": peak_src,
            "lp_gteps": ed / (ms * 1e-3) / 1e9}
    l0 = next((e for e in lp if e["name"] == "lp_persistent_level0"), None)
    if l0:
        a0 = l0["bytes"] / (l0["ms"] * 1e-3) / 1e9
        roof["level0"] = {"kernel": "k_lp, level-0 coarsening launch", "achieved": a0, "frac": a0 / peak,
                          "launches": l0["launches"], "ms_per_launch": l0["ms"] / l0["launches"],
                          "bytes_per_launch": l0["bytes"] / l0["launches"],
                          "lp_gteps": l0["edges"] / (l0["ms"] * 1e-3) / 1e9,
                          "traffic": lp_traffic(args.workload, "level0_traffic_bytes_per_launch")}
    roof["kernels_ms_per_step"] = {e["name"]: e["ms"] / args.steps for e in prof
                                   if e["launches"] > 0 and not e["name"].startswith("lp_phase")}
    roof["kernels_achieved_gbs"] = {e["name"]: {"gbs": e["bytes"] / (e["ms"] * 1e-3) / 1e9,
                                                "frac": e["bytes"] / (e["ms"] * 1e-3) / 1e9 / peak}
                                    for e in prof if e["launches"] > 0 and e["bytes"] > 0 and e["ms"] > 0}
    roof["lp_phases_ms_per_step"] = {e["name"][9:]: e["ms"] / args.steps for e in prof
                                     if e["name"].startswith("lp_phase")}
    roof["contest_calls_per_step"] = {e["name"][11:-6]: e["items"] / args.steps for e in prof
                                      if e["name"].startswith("lp_contest")}
    return roof, ed / (ms * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    import torch
    if n_gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", 0))
        local = int(os.environ.get("LOCAL_RANK", 0))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return rank, dist.get_world_size(), local, dist
    torch.cuda.set_device(0)
    return 0, 1, 0, None


def barrier(dist):
    import torch
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


def _reduce_device(dist) -> str:
    return "cpu" if dist.get_backend() == "gloo" else "cuda"


def max_over_ranks(x: float, dist) -> float:
    """Largest value over the ranks (the slowest rank's time)."""
    import torch
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist) -> float:
    """Sum over the ranks (the work all replicas did)."""
    import torch
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------------------------- CPU oracle
# The oracle is timed on every host core at once: one worker process per core, each with its own copy
# of the sample graph(s), all started together; a step's rate is the LP edges of all workers over the
# step's wall time. Samples are bounded so that a step takes a few seconds of CPU work.
SAMPLES = {
    "rgg20": ("one full oracle partition of the workload graph itself (RGG 2^20, k=16) per core",
              lambda i: [(("rgg", 1 << 20, 12.0, 1), 16, SEED)]),
    "grid256": ("one full oracle partition of the workload graph itself (grid 256x256, k=2) per core",
                lambda i: [(("grid", 256, 256), 2, SEED)]),
    "rmat24": ("one full oracle partition (k=16) per core of an R-MAT scale-17 graph of the same generator and "
               "parameters (seed 101 + core index); a full scale-24 oracle partition takes about 20 minutes",
               lambda i: [(("rmat", 17, 16, 101 + i, False), 16, SEED)]),
    "rmat22w": ("one full oracle partition (k=64) per core of a weighted R-MAT scale-16 graph of the same generator "
                "and parameters (seed 101 + core index)",
                lambda i: [(("rmat", 16, 16, 101 + i, True), 64, SEED)]),
    "rmat26w": ("one full oracle partition (k=64) per core of a weighted R-MAT scale-16 graph of the same generator "
                "and parameters (seed 101 + core index); one oracle LP round of the scale-26 graph alone takes "
                "minutes",
                lambda i: [(("rmat", 16, 16, 101 + i, True), 64, SEED)]),
}


def _make(spec):
    import graphgen as gg
    if spec[0] == "rgg":
        return gg.rgg(spec[1], spec[2], spec[3])
    if spec[0] == "grid":
        return gg.grid(spec[1], spec[2])
    if spec[0] == "batch":
        return gg.batch_graph(gg.batch_specs(512, seed=SEED)[spec[1]])
    return gg.rmat(spec[1], spec[2], seed=spec[3], weighted=spec[4])


def _oracle_worker(conn, items):
    """Worker: builds its sample graphs, then runs one oracle partition of each per 'run' command."""
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    import oracle
    graphs = [(_make(spec), k, sd) for spec, k, sd in items]
    oracle.build()
    conn.send("ready")
    while True:
        cmd = conn.recv()
        if cmd != "run":
            break
        e, t, cut = 0, 0.0, 0
        for g, k, sd in graphs:
            t0 = time.perf_counter()
            _, res = oracle.partition(g, k, EPS, sd)
            t += time.perf_counter() - t0
            e += res.lp_edges
            cut += res.cut
        conn.send((e, t, cut))


class OraclePool:
    """One oracle worker per host core (spawned processes)."""

    def __init__(self, workload: str, cores: int | None = None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        if workload == "batch512":
            # every core takes every cores-th graph of the batch
            import graphgen as gg
            specs = gg.batch_specs(512, seed=SEED)
            per = [[(("batch", j), specs[j].k, specs[j].seed) for j in range(i, 512, self.cores)][:2]
                   for i in range(self.cores)]
            self.desc = (f"two graphs of the batch per core (graphs i and i + {self.cores}), each fully "
                         f"partitioned by the oracle with its own k and seed")
        else:
            self.desc, mk = SAMPLES[workload]
            per = [mk(i) for i in range(self.cores)]
        self.conns, self.procs = [], []
        for i in range(self.cores):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, per[i]), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"

    def step(self):
        """One sample on every core: (LP edges of all cores, wall seconds, summed CPU seconds)."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("run")
        got = [c.recv() for c in self.conns]
        wall = time.perf_counter() - t0
        return sum(g[0] for g in got), wall, sum(g[1] for g in got)

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)


def levels_report(gp, dg, k, args):
    """Level by level: one gp_lp_cluster (the partition's coarsening bound U = Lmax / 14 and 10 rounds;
    one warm-up call per level) and one gp_contract of its labels, each timed with CUDA events, with the
    LP call's phase times and hub work. Isolated vertices stay in (the partition strips them first)."""
    import torch

    class _Coarse:  # a library-owned coarse graph seen as a DeviceGraph
        def __init__(self, cg):
            self.cg, self.desc, self.n = cg, cg.desc, cg.n
            self.adj = torch.empty(1, device="cuda")

    gp.lp_set_hub_keep(args.hub_keep, 0)
    U = max(1, gp.lmax(dg.n if dg.vw is None else int(dg.vw.sum()), k, EPS) // 14)
    cur = dg
    rows = []
    for lev in range(args.levels):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for _ in range(2):  # warm-up, then the profiled call
            gp.profile_read(reset=True)
            gp.profile_enable(True)
            ev[0].record()
            labels, st = gp.lp_cluster(cur, U, 10, 1000 + lev)
            ev[1].record()
            torch.cuda.synchronize()
            prof = gp.profile_read(reset=True)
            gp.profile_enable(False)
        ev[2].record()
        cg, _ = gp.contract(cur, labels)
        ev[3].record()
        torch.cuda.synchronize()
        hub = {e["name"]: e for e in prof if e["name"] in ("lp_hub_work", "lp_hub_built")}
        row = {"level": lev, "n": cur.n, "m_dir": int(cur.desc.m_dir), "lp_ms": ev[0].elapsed_time(ev[1]),
               "rounds": st["rounds"], "moves": st["moves"], "lp_edges": st["edges"],
               "contract_ms": ev[2].elapsed_time(ev[3]),
               "hub_entries": hub.get("lp_hub_work", {}).get("edges", 0),
               "hub_entries_accumulated": hub.get("lp_hub_built", {}).get("edges", 0),
               "hub_tables_stale": hub.get("lp_hub_built", {}).get("items", 0),
               "phases_ms": {e["name"][9:]: round(e["ms"], 2) for e in prof if e["name"].startswith("lp_phase")}}
        rows.append(row)
        print(json.dumps(row), flush=True)
        cur = _Coarse(cg)
        if cg.n < 4000:
            break
    gp.lp_set_hub_keep(0, 0)
    print(json.dumps({"levels": len(rows), "lp_ms": sum(r["lp_ms"] for r in rows),
                      "contract_ms": sum(r["contract_ms"] for r in rows), "hub_keep": args.hub_keep}))


def cpu_info() -> dict:
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:  # Arm kernels print no model name in /proc/cpuinfo; lscpu decodes the part number
        try:
            import subprocess
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": __import__("platform").machine()}


def bench_reference(args, w):
    """Reference arm: the CPU oracle as it stands, on every host core, a bounded sample per step."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    pool = OraclePool(args.workload)
    try:
        for _ in range(args.warmup):
            pool.step()
        tot_e, tot_t = 0, 0.0
        for _ in range(args.steps):
            e, wall, _ = pool.step()
            tot_e += e
            tot_t += wall
    finally:
        pool.close()
    value = tot_e / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": w["desc"]},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": pool.cores, "kind": "oracle",
                             "sample": pool.desc, **cpu_info()},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------- digests
DIGESTS = os.path.join(ROOT, "tests", "golden", "fullsize_digests.json")


def _sha(*arrays) -> str:
    import hashlib
    h = hashlib.sha256()
    for a, dt in arrays:
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()


def digest_check(gp, workload, dg=None, part=None, res=None, parts=None):
    """Compares the GPU's results with the oracle's stored digests of this full-size workload."""
    if not os.path.exists(DIGESTS):
        return None
    with open(DIGESTS) as f:
        gold = json.load(f).get(workload)
    if gold is None:
        return None
    if workload == "rmat24":
        ok = _sha((part.cpu().numpy(), "<i4")) == gold["part_sha256"] and res.cut == gold["cut"]
        return {"what": "full partition (labels of every vertex, cut)", "match": bool(ok)}
    if workload == "batch512":
        bad = [i for i, (p_, g_) in enumerate(zip(parts, gold["graphs"]))
               if _sha((p_.cpu().numpy(), "<i4"))[:32] != g_["part_sha256"]]
        return {"what": "every graph's partition", "graphs": len(parts), "match": not bad, "mismatched": bad[:10]}
    if workload == "rmat26w":
        import torch
        lab, st = gp.lp_cluster(dg, gold["U"], gold["rounds"], int(gold["seed_hash"]))
        ok_lab = _sha((lab.cpu().numpy(), "<i4")) == gold["labels_sha256"]
        ok_st = all(st[k] == gold["lp_stats"][k] for k in gold["lp_stats"])
        cg, f2c = gp.contract(dg, lab)
        ok_f2c = _sha((f2c.cpu().numpy(), "<i4")) == gold["f2c_sha256"]
        h = cg.to_host()
        cg.free()
        ok_c = (h.n == gold["coarse_n"] and h.m_dir == gold["coarse_m_dir"] and
                _sha((h.off, "<i8"), (h.adj, "<i4"), (h.vw, "<i8"), (h.ew, "<i8")) == gold["coarse_sha256"])
        del lab, f2c
        torch.cuda.empty_cache()
        return {"what": "level-0 gp_lp_cluster (labels, counters) and gp_contract (map, coarse CSR) at full size",
                "match": bool(ok_lab and ok_st and ok_f2c and ok_c),
                "labels": ok_lab, "lp_stats": ok_st, "f2c": ok_f2c, "coarse_csr": ok_c}
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat26w", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-digest", action="store_true")
    ap.add_argument("--once", action="store_true", help="one untimed partition (for profiler launch lists)")
    ap.add_argument("--levels", type=int, default=0,
                    help="per-level profile instead of the bench line: this many levels of gp_lp_cluster (the "
                         "coarsening bound and rounds of a partition) and gp_contract, timed one by one")
    ap.add_argument("--hub-keep", type=int, default=0,
                    help="kept hub tables for --levels (0: default budget, -1: every hub re-accumulated every sub-round)")
    ap.add_argument("--mode", default="plain", choices=["plain", "learned"])
    ap.add_argument("--no-compare", action="store_true", help="skip the learned and batched comparisons")
    ap.add_argument("--learned-seeds", type=int, default=None,
                    help="seeds 1..S of the learned-vs-plain comparison (default 10, 1 when a partition takes > 2 s)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    w = WORKLOADS[args.workload]
    is_batch = w["kind"] == "batch"
    if args.impl == "reference":
        bench_reference(args, w)
        return

    import torch
    import paper_1710_08231_gb300 as gp

    rank, world, local, dist = dist_setup(args.gpus)
    gp.build()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()
    batch_parts = None
    if is_batch:
        specs, graphs = make_batch(w["count"])
        dgs = batch_items(gp, graphs)
        ks = [sp.k for sp in specs]
        seeds = [sp.seed + rank for sp in specs]
        big = max(range(len(graphs)), key=lambda i: graphs[i].n)
        params, _ = gp.autotune(dgs[big])
        dw, dc = params.deg_warp, params.deg_cta
        g = None
        k = None

        class _Sum:  # the batch's results summed into the fields the line reports
            pass

        def step():
            nonlocal batch_parts
            batch_parts, rs = gp.partition_batch(dgs, ks, EPS, seeds, params)
            r = _Sum()
            r.lp_edges = sum(x.lp_edges for x in rs)
            r.cut = sum(x.cut for x in rs)
            r.max_block_weight = max(x.max_block_weight for x in rs)
            r.lmax = None
            r.imbalanced = sum(x.imbalanced for x in rs)
            r.levels = max(x.levels for x in rs)
            r.level_n = None
            return r
    else:
        t_gen = time.perf_counter()
        g = make_graph(args.workload)
        t_gen = time.perf_counter() - t_gen
        k = w["k"]
        dg = gp.DeviceGraph.from_host(g)
        part = torch.empty(g.n, dtype=torch.int32, device="cuda")
        params = None
        if args.mode == "learned":
            mlp, _ = train_scorer(gp, args.workload, k)
            params = gp.default_params(mode=gp.MODE_LEARNED)
            params.mlp = mlp.data_ptr()

        def step():
            _, res = gp.partition(dg, k, EPS, SEED + rank, params, out=part)
            return res

    if args.levels:
        levels_report(gp, dg, k, args)
        return
    if args.once:
        res = step()
        torch.cuda.synchronize()
        print(json.dumps({"once": True, "cut": res.cut, "lp_edges": res.lp_edges, "launches": gp.launch_count()}))
        return

    for _ in range(args.warmup):
        res0 = step()
    lp_edges_step = res0.lp_edges

    # ---- pass A: the timed region (device time per step, L2 flushed between steps). The library's
    # per-launch CUDA events (on the launching stream) give each kernel's time inside this region.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = gp.launch_count()
    gp.profile_read(reset=True)
    gp.profile_enable(True)
    barrier(dist)
    with ClockSampler(torch.cuda.current_device()) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            res = step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(dist)
    gp.profile_enable(False)
    prof = gp.profile_read(reset=True)
    launches = gp.launch_count() - launches0
    ms_local = sum(a.elapsed_time(b) for a, b in ev)
    ms_total = max_over_ranks(ms_local, dist)
    edges_all = sum_over_ranks(float(lp_edges_step * args.steps), dist)
    value = edges_all / (ms_total * 1e-3) / 1e9
    ms_step = ms_total / args.steps

    peak, peak_kind = peaks()
    roofline, lp_only = lp_roofline(prof, args, peak, peak_kind)

    digest = None
    if rank == 0 and not args.no_digest:
        digest = digest_check(gp, args.workload, dg=None if is_batch else dg, part=None if is_batch else part,
                              res=res, parts=batch_parts)

    # ---- pass B: end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    e2e_steps = args.steps if ms_step < 2000 else min(args.steps, 3)
    if not args.no_e2e and is_batch:
        # host CSR in pinned memory; every step copies all graphs in, partitions, copies the parts out
        hosts = [(torch.from_numpy(np.ascontiguousarray(x.off)).pin_memory(),
                  torch.from_numpy(np.ascontiguousarray(x.adj)).pin_memory()) for x in graphs]
        outs = [torch.empty(x.n, dtype=torch.int32).pin_memory() for x in graphs]
        h2d = sum(a.numel() * a.element_size() + b.numel() * b.element_size() for a, b in hosts)
        d2h = sum(o.numel() * 4 for o in outs)

        def e2e_step():
            devs = [gp.DeviceGraph(x.n, a.to("cuda", non_blocking=True), b.to("cuda", non_blocking=True), None, None)
                    for x, (a, b) in zip(graphs, hosts)]
            parts, rs = gp.partition_batch(devs, ks, EPS, seeds, params)
            for p_, o in zip(parts, outs):
                o.copy_(p_, non_blocking=True)
            torch.cuda.synchronize()
            return rs

        e2e_step()
        barrier(dist)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            e2e_step()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": lp_edges_step * world * e2e_steps / e2e_s / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s / e2e_steps, "steps": e2e_steps}
    elif not args.no_e2e and params is None:
        hg = gp.HostGraph(g, pin=True)
        gp.partition_host(hg, k, EPS, SEED + rank)
        barrier(dist)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            gp.partition_host(hg, k, EPS, SEED + rank)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": lp_edges_step * world * e2e_steps / e2e_s / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": hg.h2d_bytes, "d2h_bytes_per_step": hg.d2h_bytes,
               "ms_per_step": 1e3 * e2e_s / e2e_steps, "steps": e2e_steps}
        del hg

    compare = None
    if rank == 0 and world == 1 and not args.no_compare and not is_batch and args.mode == "plain":
        nseeds = args.learned_seeds if args.learned_seeds is not None else (10 if ms_step < 2000 else 1)
        compare = {"learned": compare_learned(gp, args.workload, g, dg, k, min(args.steps, 3), flush, ms_step, res,
                                              nseeds),
                   "batched": compare_batched(gp, 3, flush),
                   "ip_tries": compare_ip_tries(gp, args.workload, dg, k, ms_step, flush),
                   "variants": compare_variants(gp, args.workload, dg, k, ms_step, flush)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(args.workload)
        try:
            e, wall_c, cpu_s = pool.step()
        finally:
            pool.close()
        cpu = {"value": e / wall_c / 1e9, "unit": "GTEPS", "cores": pool.cores, "kind": "oracle",
               "sample": pool.desc + f" ({wall_c:.1f} s wall, {cpu_s:.0f} s CPU)", **cpu_info()}

    if rank == 0:
        shape = ({"graphs": len(graphs), "n_total": int(sum(x.n for x in graphs)),
                  "m_dir_total": int(sum(x.m_dir for x in graphs)), "k": "2, 4 or 8 per graph",
                  "schedule": {"deg_warp": dw, "deg_cta": dc, "verts_per_block": params.verts_per_block,
                               "hub_batch_slots": params.hub_batch_slots,
                               "picked_by": "gp_autotune on the largest graph"}}
                 if is_batch else {"n": g.n, "m_dir": g.m_dir, "k": k, "mode": args.mode,
                                   "generation_s": round(t_gen, 1)})
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": w["desc"], **shape,
                           "lp_edges_per_partition": lp_edges_step, "cut": res.cut,
                           "max_block_weight": res.max_block_weight, "lmax": res.lmax,
                           "imbalanced": res.imbalanced, "levels": res.levels,
                           "level_n": res.level_n, "ms_per_partition": ms_step,
                           "lp_only_gteps": lp_only,
                           "l2": "flushed between steps (256 MB write outside the per-step events); inputs "
                                 + ("larger than L2" if (is_batch or g.m_dir * 4 > 129e6) else "smaller than L2"),
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "wall_ms_per_step": 1e3 * wall / args.steps},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "oracle_digest_match": digest, "compare": compare}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
