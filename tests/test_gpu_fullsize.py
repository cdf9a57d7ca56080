"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

* Random geometric graph, 2^20 vertices, average degree 12, k=16 (the default bench workload): the
  whole partition is compared element by element with the oracle (about 4 s of oracle time).
* R-MAT scale 24 (16.7M vertices, 521M CSR entries), k=16: the whole partition against the oracle's
  stored digest (tests/golden/fullsize_digests.json, written by make_fullsize_digests.py, which calls
  only the oracle; its run takes about 20 minutes), plus properties that hold at any size, recomputed
  on the host from the input graph: every block id in [0, k), the reported cut equals the cut of the
  returned partition, the reported block weights and balance match, degree-0 vertices are placed, and
  every level is smaller than the one before.
* The batch of 512 uneven graphs with default parameters, in one gp_partition_batch call: every
  graph's partition against the oracle's stored digest.
* R-MAT scale 26 with edge weights (the largest configuration): level-0 gp_lp_cluster and gp_contract
  at full size against the oracle's stored digests of labels, counters, map and coarse CSR.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1710_08231_gb300 as m
    m.build()
    m.lp_set_schedule(0, 0)
    return m


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_digests.json")


def _gold(key):
    data = json.load(open(GOLDEN)) if os.path.exists(GOLDEN) else {}
    if key not in data:
        pytest.fail(f"{GOLDEN} has no entry {key}: run tests/golden/make_fullsize_digests.py {key}")
    return data[key]


def _sha(*arrays):
    h = hashlib.sha256()
    for a, dt in arrays:
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()


def _host_cut(g, part):
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off))
    cross = part[src] != part[g.adj]
    w = np.ones(g.m_dir, dtype=np.int64) if g.ew is None else g.ew.astype(np.int64)
    return int(w[cross].sum()) // 2


def _host_block_weights(g, part, k):
    vw = np.ones(g.n, dtype=np.int64) if g.vw is None else g.vw.astype(np.int64)
    return np.bincount(part, weights=vw, minlength=k).astype(np.int64)


def test_rgg_2e20_k16_bit_exact_with_oracle(gp):
    g = gg.rgg(1 << 20, 12.0, 1)
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, 16, 0.03, 1)
    p = part.cpu().numpy()
    po, ro = O.partition(g, 16, 0.03, 1)
    assert np.array_equal(p, po)
    assert (res.cut, res.levels, res.best_try, res.n_isolated) == (ro.cut, ro.levels, ro.best_try, ro.n_isolated)
    assert res.level_n == list(ro.level_n[: ro.levels + 1])
    assert res.lp_edges == ro.lp_edges


def test_rmat_scale24_k16_properties(gp):
    g = gg.rmat(24, 16, seed=1)
    dg = gp.DeviceGraph.from_host(g)
    k = 16
    part, res = gp.partition(dg, k, 0.03, 1)
    p = part.cpu().numpy()
    assert p.shape == (g.n,) and p.min() >= 0 and p.max() < k
    assert res.cut == _host_cut(g, p)
    bw = _host_block_weights(g, p, k)
    assert res.max_block_weight == int(bw.max())
    assert res.lmax == O.lmax(g.n, k, 0.03)
    assert res.imbalanced == int(bw.max() > res.lmax)
    assert res.n_isolated == int((np.diff(g.off) == 0).sum())
    assert all(a > b for a, b in zip(res.level_n[:-1], res.level_n[1:]))
    # the same call again gives the same partition (deterministic at full size)
    part2, res2 = gp.partition(dg, k, 0.03, 1)
    assert np.array_equal(p, part2.cpu().numpy()) and res2.cut == res.cut
    # bit-exact with the oracle's full partition
    gold = _gold("rmat24")
    assert (g.n, g.m_dir) == (gold["n"], gold["m_dir"])
    assert _sha((p, "<i4")) == gold["part_sha256"]
    assert (res.cut, res.max_block_weight, res.levels, res.best_try, res.lp_edges, res.n_isolated) == (
        gold["cut"], gold["max_block_weight"], gold["levels"], gold["best_try"], gold["lp_edges"], gold["n_isolated"])
    assert res.level_n == gold["level_n"] and res.level_m == gold["level_m"]


def test_batch512_default_params_bit_exact_with_oracle(gp):
    gold = _gold("batch512")["graphs"]
    specs = gg.batch_specs(512, seed=1)
    graphs = [gg.batch_graph(sp) for sp in specs]
    dgs = [gp.DeviceGraph.from_host(g) for g in graphs]
    parts, results = gp.partition_batch(dgs, [sp.k for sp in specs], 0.03, [sp.seed for sp in specs])
    bad = []
    for i, (p, r, gd) in enumerate(zip(parts, results, gold)):
        if _sha((p.cpu().numpy(), "<i4"))[:32] != gd["part_sha256"] or r.cut != gd["cut"] or \
                r.imbalanced != gd["imbalanced"]:
            bad.append(i)
    assert not bad, f"graphs differing from the oracle: {bad[:20]}"


def test_rmat26_weighted_level0_cluster_and_contract_bit_exact_with_oracle(gp):
    gold = _gold("rmat26w")
    g = gg.rmat(26, 16, seed=1, weighted=True)
    assert (g.n, g.m_dir) == (gold["n"], gold["m_dir"])
    dg = gp.DeviceGraph.from_host(g)
    del g
    lab, st = gp.lp_cluster(dg, gold["U"], gold["rounds"], int(gold["seed_hash"]))
    assert _sha((lab.cpu().numpy(), "<i4")) == gold["labels_sha256"]
    assert {k: st[k] for k in gold["lp_stats"]} == gold["lp_stats"]
    cg, f2c = gp.contract(dg, lab)
    assert _sha((f2c.cpu().numpy(), "<i4")) == gold["f2c_sha256"]
    assert (cg.n, cg.m_dir) == (gold["coarse_n"], gold["coarse_m_dir"])
    h = cg.to_host()
    cg.free()
    assert _sha((h.off, "<i8"), (h.adj, "<i4"), (h.vw, "<i8"), (h.ew, "<i8")) == gold["coarse_sha256"]
