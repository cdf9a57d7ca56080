"""Batched partitioning: every graph of a batch equals gp_partition on that graph alone and the oracle.

The batch mixes grids and random geometric graphs of uneven sizes (the batched workload's families),
an R-MAT graph with degree-0 vertices and a weighted graph."""
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


def _batch():
    specs = gg.batch_specs(10, seed=5, n_lo=400, n_hi=30000)
    graphs = [gg.batch_graph(s) for s in specs]
    ks = [s.k for s in specs]
    seeds = [s.seed for s in specs]
    graphs.append(gg.rmat(11, 8, seed=3))               # degree-0 vertices, hubs
    ks.append(8)
    seeds.append(17)
    graphs.append(gg.rmat(10, 8, seed=4, weighted=True))  # edge weights
    ks.append(4)
    seeds.append(18)
    return graphs, ks, seeds


def _params(gp, **kw):
    p = gp.default_params(coarse_min=300, **kw)
    return p


def test_batch_equals_single_and_oracle(gp):
    graphs, ks, seeds = _batch()
    dgs = [gp.DeviceGraph.from_host(g) for g in graphs]
    parts, results = gp.partition_batch(dgs, ks, 0.03, seeds, _params(gp))
    op = O.default_params()
    op.coarse_min = 300
    for g, dg, k, sd, pb, rb in zip(graphs, dgs, ks, seeds, parts, results):
        ps, rs = gp.partition(dg, k, 0.03, sd, _params(gp))
        assert np.array_equal(pb.cpu().numpy(), ps.cpu().numpy())
        assert (rb.cut, rb.levels, rb.best_try, rb.n_isolated, rb.max_block_weight) == \
               (rs.cut, rs.levels, rs.best_try, rs.n_isolated, rs.max_block_weight)
        assert rb.level_n == rs.level_n and rb.level_m == rs.level_m and rb.try_cut == rs.try_cut
        assert rb.lp_edges == rs.lp_edges
        if g.n <= 40000:
            po, ro = O.partition(g, k, 0.03, sd, op)
            assert np.array_equal(pb.cpu().numpy(), po) and rb.cut == ro.cut


def test_batch_schedule_invariance(gp):
    graphs, ks, seeds = _batch()
    dgs = [gp.DeviceGraph.from_host(g) for g in graphs]
    a, ra = gp.partition_batch(dgs, ks, 0.03, seeds, _params(gp))
    b, rb = gp.partition_batch(dgs, ks, 0.03, seeds, _params(gp, deg_warp=32, deg_cta=64))
    for x, y, r1, r2 in zip(a, b, ra, rb):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy()) and r1.cut == r2.cut


def test_autotuner_returns_a_candidate_and_results_do_not_change(gp):
    g = gg.rmat(13, 16, seed=8)
    dg = gp.DeviceGraph.from_host(g)
    w, c, ms = gp.autotune_schedule(dg)
    assert (w, c) in [(32, 256), (64, 256), (64, 512), (128, 512), (128, 1024), (32, 1024), (128, 2048),
                      (256, 2048)] and ms > 0
    p0, r0 = gp.partition(dg, 16, 0.03, 3)
    p1, r1 = gp.partition(dg, 16, 0.03, 3, gp.default_params(deg_warp=w, deg_cta=c))
    assert np.array_equal(p0.cpu().numpy(), p1.cpu().numpy())
