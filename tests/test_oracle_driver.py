"""Pins of the oracle's multilevel driver (``oracle.partition``).

The primitives the driver composes -- LP (clustering and refinement), contraction, bisection,
repair, cut -- are pinned by tests/test_oracle.py against hand traces and brute force. This file pins
the composition itself, which no primitive test sees:

* the stop rule of coarsening: n <= T = max(coarse_min, coarse_per_k * k) with T reached exactly and
  missed by one vertex, the stall rule (a contraction that keeps more than stall_pct % of the vertices
  ends coarsening and that level is kept), and the cap on the number of contractions;
* the seeds of every phase: coarsening LP at level l with H(seed, l, 1), refinement at level l with
  H(seed, l, 2), try t on the coarsest level c with s_try = H(seed, c, 4 + t) and its refinement with
  H(s_try, c, 3);
* the choice of the initial-partitioning try: the minimum of (cut, imbalanced, t);
* projection: level l's partition is the coarser level's partition read through level l's map, and
  it has the coarse partition's cut and block weights (Section III-A: the quotient graph keeps cut and
  balance of a partition that does not split clusters);
* degree-0 vertices: removed before coarsening with ids re-ranked, placed last;
* the options: matching instead of LP clustering, and multi-try local search after every level's
  LP refinement (seed H(seed, l, 7)).

The check restates the multilevel scheme of Sections III and IV step by step in Python, calling only
the pinned primitives, exposes every intermediate value (tests/golden/partition_trace.json records
one such trace, written by make_partition_trace.py), and requires the driver's result to equal it on
many graphs and parameter sets. A driver that used a wrong seed phase, stopped one level early or
late, kept the worst try or projected through the wrong level's map fails it.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = 0.03


def restated_partition(g, k, eps, seed, p=None, trace=None):
    """The multilevel scheme of Sections III-IV with this repository's readings, from the primitives."""
    p = p or O.default_params()
    n = g.n
    vw = O.vertex_weights(g)
    W = int(vw.sum())
    lmax = O.lmax(W, k, eps)
    deg = np.diff(g.off)
    keep = np.flatnonzero(deg > 0)
    rank = -np.ones(n, dtype=np.int64)
    rank[keep] = np.arange(len(keep))
    # level 0: the graph induced by vertices of degree > 0, ids by rank (row order kept)
    off0 = np.concatenate([[0], np.cumsum(deg[keep])]).astype(np.int64)
    adj0 = rank[g.adj].astype(np.int32)
    ew0 = None if g.ew is None else np.asarray(g.ew, dtype=np.int64)
    G = [gg.Graph(len(keep), off0, adj0, vw[keep].astype(np.int64), ew0)]
    maps = []
    lp_edges = 0
    T = max(p.coarse_min, p.coarse_per_k * k)
    t = trace if trace is not None else {}
    t.update({"lmax": lmax, "T": T, "levels": []})
    cur = None
    if G[0].n > 0:
        while G[-1].n > T and len(maps) < p.max_levels:
            lvl = len(maps)
            gl = G[-1]
            U = max(int(gl.vw.max()), lmax // p.cluster_div)
            s1 = O.hash3(seed, lvl, 1)
            if p.coarsen_mode == 1:  # matching-based clustering
                labels, _ = O.match(gl, U, p.rounds_coarsen, s1)
            else:
                labels, _, st = O.lp_cluster(gl, U, p.rounds_coarsen, s1)
                lp_edges += st.edges
            gc, f2c = O.contract(gl, labels)
            t["levels"].append({"n": gl.n, "m_dir": gl.m_dir, "U": U, "seed": s1, "coarse_n": gc.n})
            G.append(gc)
            maps.append(f2c)
            if 100 * gc.n > p.stall_pct * gl.n:
                break
        c = len(maps)
        gc = G[-1]
        tries = []
        for tr in range(p.ip_tries):
            s_try = O.hash3(seed, c, 4 + tr)
            pt = O.bisect(gc, k, s_try)
            pt, _ = O.repair(gc, pt, k, lmax, p.repair_rounds)
            pt, bw, st = O.lp_refine(gc, pt, k, lmax, p.rounds_refine, O.hash3(s_try, c, 3))
            lp_edges += st.edges
            cut, bw2 = O.cut(gc, pt, k)
            assert np.array_equal(bw, bw2)
            tries.append((cut, int(bw.max() > lmax), tr, pt))
        best = min(tries, key=lambda x: (x[0], x[1], x[2]))
        t["tries"] = [{"s_try": O.hash3(seed, c, 4 + tr), "cut": x[0], "imbalanced": x[1]}
                      for tr, x in enumerate(tries)]
        t["best_try"] = best[2]
        cur = best[3]
        mp = O.mls_default_params()
        mp.global_iters = p.mls
        if p.mls:  # multi-try local search after the coarsest level's refinement
            cur, _ = O.mls(gc, cur, k, lmax, O.hash3(seed, c, 7), mp)
        t["uncoarsen"] = []
        for lvl in range(c - 1, -1, -1):
            fine = cur[maps[lvl]]
            # projection keeps the cut and the block weights
            cc, bwc = O.cut(G[lvl + 1], cur, k)
            cf, bwf = O.cut(G[lvl], fine, k)
            assert cc == cf and np.array_equal(bwc, bwf)
            fine, _, st = O.lp_refine(G[lvl], fine, k, lmax, p.rounds_refine, O.hash3(seed, lvl, 2))
            lp_edges += st.edges
            if p.mls:
                fine, _ = O.mls(G[lvl], fine, k, lmax, O.hash3(seed, lvl, 7), mp)
            t["uncoarsen"].append({"level": lvl, "projected_cut": cf, "refined_cut": O.cut(G[lvl], fine, k)[0]})
            cur = fine
    part = np.zeros(n, dtype=np.int32)
    bw = np.zeros(k, dtype=np.int64)
    if cur is not None:
        part[keep] = cur
        np.add.at(bw, cur, vw[keep])
    for v in np.flatnonzero(deg == 0):  # ascending id, each to the lightest block (smaller id on ties)
        b = int(np.argmin(bw))
        part[v] = b
        bw[b] += vw[v]
    t.update({"cut": O.cut(g, part, k)[0], "lp_edges": lp_edges, "level_n": [x.n for x in G],
              "level_m": [x.m_dir for x in G]})
    return part, t


def _check(g, k, seed, p=None):
    part, t = restated_partition(g, k, EPS, seed, p)
    po, ro = O.partition(g, k, EPS, seed, p)
    assert ro.levels == len(t["levels"])
    assert list(ro.level_n[: ro.levels + 1]) == t["level_n"]
    assert list(ro.level_m[: ro.levels + 1]) == t["level_m"]
    if "tries" in t:
        assert list(ro.try_cut[: len(t["tries"])]) == [x["cut"] for x in t["tries"]]
        assert list(ro.try_imbalanced[: len(t["tries"])]) == [x["imbalanced"] for x in t["tries"]]
        assert ro.best_try == t["best_try"]
    assert ro.lp_edges == t["lp_edges"]
    assert np.array_equal(po, part)
    assert ro.cut == t["cut"] and ro.lmax == t["lmax"]
    return t, ro


def _params(**kw):
    p = O.default_params()
    for a, v in kw.items():
        setattr(p, a, v)
    return p


def _with_isolated(g, extra):
    """g plus `extra` degree-0 vertices interleaved (every third id)."""
    n2 = g.n + extra
    iso = set(range(1, 3 * extra, 3))
    old = [v for v in range(n2) if v not in iso][: g.n]
    new_id = np.array(old, dtype=np.int64)
    deg = np.zeros(n2, dtype=np.int64)
    deg[new_id] = np.diff(g.off)
    off = np.concatenate([[0], np.cumsum(deg)])
    adj = new_id[g.adj].astype(np.int32)
    return gg.Graph(n2, off, adj, None, g.ew)


CASES = [
    ("grid24x24_k2", lambda: gg.grid(24, 24), 2, dict(coarse_min=60)),
    ("grid17x29_k3", lambda: gg.grid(17, 29), 3, dict(coarse_min=40, coarse_per_k=8)),
    ("rgg3000_k8", lambda: gg.rgg(3000, 9.0, 7), 8, dict(coarse_min=100, coarse_per_k=8)),
    ("rmat11_k4", lambda: gg.rmat(11, 8, seed=9), 4, dict(coarse_min=150)),
    ("rmat10w_k5", lambda: gg.rmat(10, 8, seed=2, weighted=True), 5, dict(coarse_min=80, ip_tries=7)),
    ("rgg2000_iso_k4", lambda: _with_isolated(gg.rgg(2000, 8.0, 3), 50), 4, dict(coarse_min=90)),
    ("grid30x30_norefine", lambda: gg.grid(30, 30), 4, dict(coarse_min=50, rounds_refine=0, repair_rounds=0)),
    ("rgg4000_default", lambda: gg.rgg(4000, 10.0, 11), 2, dict()),
    ("grid40x40_matching", lambda: gg.grid(40, 40), 4, dict(coarse_min=100, coarsen_mode=1)),
    ("rmat11_matching", lambda: gg.rmat(11, 8, seed=9), 4, dict(coarse_min=150, coarsen_mode=1)),
    ("rgg3000_mls", lambda: gg.rgg(3000, 9.0, 7), 8, dict(coarse_min=100, coarse_per_k=8, mls=3)),
    ("grid30x30_mls_matching", lambda: gg.grid(30, 30), 4, dict(coarse_min=50, mls=2, coarsen_mode=1)),
]


@pytest.mark.parametrize("name,make,k,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("seed", [1, 12345])
def test_driver_equals_restated_scheme(name, make, k, kw, seed):
    t, ro = _check(make(), k, seed, _params(**kw))
    if kw.get("coarse_min", 2000) < 2000 and name != "rgg4000_default":
        assert ro.levels >= 1  # the cases are chosen so that coarsening happens


def test_stop_rule_at_T_exactly_and_one_above():
    # a path of T vertices is not coarsened; T + 1 vertices are (T = coarse_min here)
    for n, want_levels in [(40, 0), (41, 1)]:
        edges = [(i, i + 1) for i in range(n - 1)]
        g = _path(n)
        p = _params(coarse_min=40, coarse_per_k=1, max_levels=1)
        t, ro = _check(g, 2, 3, p)
        assert ro.levels == want_levels
    # T comes from coarse_per_k * k when that is larger
    g = gg.grid(10, 10)
    t, ro = _check(g, 4, 3, _params(coarse_min=10, coarse_per_k=25))  # T = 100 = n
    assert ro.levels == 0
    t, ro = _check(g, 4, 3, _params(coarse_min=10, coarse_per_k=24))  # T = 96 < n
    assert ro.levels >= 1


def _path(n):
    off = np.concatenate([[0], np.cumsum([1] + [2] * (n - 2) + [1])]).astype(np.int64)
    adj = []
    for v in range(n):
        if v > 0:
            adj.append(v - 1)
        if v < n - 1:
            adj.append(v + 1)
    return gg.Graph(n, off, np.array(adj, dtype=np.int32))


def test_stall_rule_keeps_the_stalled_level():
    # cluster_div so large that U = max c(v) = 1: no vertex can join another, the contraction keeps
    # every vertex, coarsening stops after that one level and the level is kept
    g = gg.grid(20, 20)
    t, ro = _check(g, 2, 5, _params(coarse_min=50, cluster_div=10**9))
    assert ro.levels == 1 and ro.level_n[1] == ro.level_n[0] == 400
    # with stall_pct 100 a stall would need n' > n, which never happens: coarsening goes on to T
    t, ro = _check(g, 2, 5, _params(coarse_min=20, coarse_per_k=1, stall_pct=100, max_levels=6))
    assert ro.levels == 6 or ro.level_n[ro.levels] <= 20


def test_level_cap():
    g = gg.rgg(6000, 10.0, 4)
    for cap in (0, 1, 2):
        t, ro = _check(g, 2, 8, _params(coarse_min=20, max_levels=cap))
        assert ro.levels == cap


def test_try_selection_ties():
    """Across small instances with uneven vertex weights, some tries tie on the cut and differ in
    balance, and some tie on both: the driver must keep the balanced one, then the first."""
    tie_imb = tie_both = 0
    for s in range(1, 60):
        g = gg.grid(4 + s % 4, 5 + s % 3)
        g.vw = np.random.default_rng(s).integers(1, 9, g.n).astype(np.int64)
        p = _params(coarse_min=1000, rounds_refine=0 if s % 2 else 25, repair_rounds=0 if s % 3 else 16,
                    ip_tries=16)
        t, ro = _check(g, 2 + s % 4, s, p)
        tries = [(x["cut"], x["imbalanced"]) for x in t["tries"]]
        best = tries[ro.best_try]
        assert all(x >= best for x in tries)
        if any(c == best[0] and i > best[1] for c, i in tries):
            tie_imb += 1
        if any(j < ro.best_try for j, x in enumerate(tries) if x == best):
            raise AssertionError("an earlier try with equal (cut, imbalanced) must be kept")
        if sum(1 for x in tries if x == best) > 1:
            tie_both += 1
    assert tie_imb > 0 and tie_both > 0


def test_partition_trace_golden():
    """tests/golden/partition_trace.json: one full trace (levels, bounds, seeds, every try, every
    projection) written by make_partition_trace.py; the driver's reported values must equal it."""
    with open(os.path.join(GOLD, "partition_trace.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        g = _path(case["path_n"]) if "path_n" in case else gg.grid(case["grid"][0], case["grid"][1])
        p = _params(**case["params"])
        po, ro = O.partition(g, case["k"], EPS, case["seed"], p)
        tr = case["trace"]
        assert ro.levels == len(tr["levels"])
        assert list(ro.level_n[: ro.levels + 1]) == tr["level_n"]
        assert [x["cut"] for x in tr["tries"]] == list(ro.try_cut[: len(tr["tries"])])
        assert ro.best_try == tr["best_try"] and ro.cut == tr["cut"] and ro.lp_edges == tr["lp_edges"]
        assert [int(x) for x in po] == case["part"]
        if case.get("grid") == [4, 6]:
            # by hand: the two halves of three columns each, the minimum bisection of a 4 x 6 grid
            assert ro.cut == 4 and all(po[r * 6 + c] == po[0] for r in range(4) for c in range(3))
        # the recorded seeds are the hash phases of the readings
        for lvl, rec in enumerate(tr["levels"]):
            assert int(rec["seed"]) == O.hash3(case["seed"], lvl, 1)
        for tno, rec in enumerate(tr["tries"]):
            assert int(rec["s_try"]) == O.hash3(case["seed"], len(tr["levels"]), 4 + tno)
