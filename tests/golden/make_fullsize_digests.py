"""Writes tests/golden/fullsize_digests.json: the oracle's results on the full-size configurations,
reduced to SHA-256 digests, so that GPU tests and the benchmark can check bit-exact parity at sizes
whose oracle run takes minutes to hours (the oracle is run here once, never on the GPU path).

Calls only ``oracle`` (the CPU oracle) and ``graphgen`` (the seeded input generator).

    python tests/golden/make_fullsize_digests.py rmat24      # R-MAT scale 24, k=16: full partition
    python tests/golden/make_fullsize_digests.py rmat26w     # R-MAT scale 26 weighted: level-0 LP + contraction
    python tests/golden/make_fullsize_digests.py batch512    # the 512-graph batch: every graph's partition

Digest of an array: sha256 of its little-endian bytes (int32 for labels, maps and partitions; the
coarse CSR as int64 offsets, int32 adjacency, int64 vertex and edge weights, concatenated).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "fullsize_digests.json")
EPS = 0.03


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a, dt in arrays:
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()


def partition_entry(g, k, seed, part, res) -> dict:
    return {"n": int(g.n), "m_dir": int(g.m_dir), "k": k, "seed": seed, "part_sha256": sha((part, "<i4")),
            "cut": int(res.cut), "max_block_weight": int(res.max_block_weight), "lmax": int(res.lmax),
            "imbalanced": int(res.imbalanced), "levels": int(res.levels),
            "level_n": [int(x) for x in res.level_n[: res.levels + 1]],
            "level_m": [int(x) for x in res.level_m[: res.levels + 1]], "best_try": int(res.best_try),
            "lp_edges": int(res.lp_edges), "n_isolated": int(res.n_isolated)}


def do_rmat24() -> dict:
    import graphgen as gg
    import oracle as O
    g = gg.rmat(24, 16, seed=1)
    t0 = time.time()
    part, res = O.partition(g, 16, EPS, 1)
    e = partition_entry(g, 16, 1, part, res)
    e["oracle_s"] = round(time.time() - t0, 1)
    e["config"] = "R-MAT scale 24, edge factor 16, (0.57,0.19,0.19), unit weights, k=16, eps=0.03, seed 1"
    return e


def level0_params(n: int, k: int, seed: int):
    """U and seed of a partition's level-0 coarsening LP with default parameters and unit vertex weights
    (U = max(max c(v), floor(Lmax / 14)), seed H(seed, 0, 1))."""
    import oracle as O
    return max(1, O.lmax(n, k, EPS) // 14), O.hash3(seed, 0, 1)


def do_rmat26w() -> dict:
    import ctypes

    import graphgen as gg
    import oracle as O
    g = gg.rmat(26, 16, seed=1, weighted=True)
    n, m = g.n, g.m_dir
    U, s1 = level0_params(n, 64, 1)
    # one int64 copy of the edge weights (the oracle's width) instead of the int32 array plus a copy
    g.ew = g.ew.astype(np.int64)
    t0 = time.time()
    labels, _, st = O.lp_cluster(g, U, 10, s1)
    t_lp = time.time() - t0
    out = {"n": n, "m_dir": m, "U": U, "rounds": 10, "seed_hash": str(s1),
           "labels_sha256": sha((labels, "<i4")),
           "lp_stats": {"rounds": st.rounds, "moves": st.moves, "visits": st.visits, "edges": st.edges,
                        "movers": st.movers}, "oracle_lp_s": round(t_lp, 1)}
    # contraction with output buffers sized by the cut entries (an upper bound of the coarse entries)
    cut_entries = 0
    step = 1 << 22
    for v0 in range(0, n, step):
        v1 = min(n, v0 + step)
        a, b = int(g.off[v0]), int(g.off[v1])
        src = np.repeat(labels[v0:v1], np.diff(g.off[v0:v1 + 1]))
        cut_entries += int(np.count_nonzero(src != labels[g.adj[a:b]]))
    view = O._View(g)
    L = O._load()
    off = np.zeros(n + 1, dtype=np.int64)
    cadj = np.zeros(max(cut_entries, 1), dtype=np.int32)
    cvw = np.zeros(n, dtype=np.int64)
    cew = np.zeros(max(cut_entries, 1), dtype=np.int64)
    f2c = np.zeros(n, dtype=np.int32)
    nn, mm = ctypes.c_int64(0), ctypes.c_int64(0)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    t0 = time.time()
    rc = L.or_contract(view.ref(), lab.ctypes.data, n, ctypes.byref(nn), ctypes.byref(mm), off.ctypes.data,
                       cadj.ctypes.data, cvw.ctypes.data, cew.ctypes.data, f2c.ctypes.data)
    assert rc == 0
    n2, m2 = nn.value, mm.value
    out.update({"f2c_sha256": sha((f2c, "<i4")), "coarse_n": int(n2), "coarse_m_dir": int(m2),
                "coarse_sha256": sha((off[: n2 + 1], "<i8"), (cadj[:m2], "<i4"), (cvw[:n2], "<i8"),
                                     (cew[:m2], "<i8")),
                "oracle_contract_s": round(time.time() - t0, 1),
                "config": "R-MAT scale 26, edge factor 16, edge weights 1 + (key & 7), seed 1: gp_lp_cluster "
                          "with the level-0 U and seed of a k=64, eps=0.03, seed-1 partition, then gp_contract"})
    return out


def _batch_one(i):
    import graphgen as gg
    import oracle as O
    sp = gg.batch_specs(512, seed=1)[i]
    g = gg.batch_graph(sp)
    part, res = O.partition(g, sp.k, EPS, sp.seed)
    return i, {"k": sp.k, "n": int(g.n), "cut": int(res.cut), "imbalanced": int(res.imbalanced),
               "part_sha256": sha((part, "<i4"))[:32]}


def do_batch512() -> dict:
    import multiprocessing as mp
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        got = dict(pool.map(_batch_one, range(512), chunksize=4))
    return {"graphs": [got[i] for i in range(512)], "oracle_s": round(time.time() - t0, 1),
            "config": "batch of 512 graphs (graphgen.batch_specs(512, seed=1)), each partitioned alone with its "
                      "own k and seed, eps=0.03"}


def main():
    which = sys.argv[1:] or ["batch512", "rmat24", "rmat26w"]
    for w in which:
        t0 = time.time()
        entry = {"rmat24": do_rmat24, "rmat26w": do_rmat26w, "batch512": do_batch512}[w]()
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[w] = entry
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(f"{w}: done in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
