"""GPU matching-based clustering (gp_match) and matching-coarsened partitions against the oracle,
element by element: labels, rounds and pairs of the matching, and the whole partition with
coarsen = GP_COARSEN_MATCHING (every level matched, contracted, refined).

Graphs: meshes (grids, random geometric graphs: the family the matching is meant for), weighted
vertices and edges (the rating omega^2 / (c(u) c(v)) and the bound U decide), and R-MAT graphs whose
vertices of degree above 256 take the one-CTA-per-vertex proposal kernel."""
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
    return m


def _weighted_rgg(n, seed):
    g = gg.rgg(n, 7.0, seed)
    rng = np.random.default_rng(seed)
    g.vw = rng.integers(1, 6, g.n).astype(np.int32)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    lo, hi = np.minimum(src, g.adj), np.maximum(src, g.adj)
    g.ew = (1 + (lo * 7919 + hi * 104729) % 9).astype(np.int32)
    return g


GRAPHS = {
    "grid128": lambda: gg.grid(128, 128),
    "grid_ragged": lambda: gg.grid(37, 53),
    "rgg2e15": lambda: gg.rgg(1 << 15, 8.0, 2),
    "rgg_weighted": lambda: _weighted_rgg(20000, 5),
    "rmat14": lambda: gg.rmat(14, 16, seed=3),
    "rmat12w": lambda: gg.rmat(12, 16, seed=4, weighted=True),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("rounds,U", [(1, 2), (3, 4), (1000, 2), (1000, 9)])
def test_match_equals_oracle(gp, name, rounds, U):
    g = GRAPHS[name]()
    U = max(U, int(O.vertex_weights(g).max()))
    dg = gp.DeviceGraph.from_host(g)
    lab, st = gp.match(dg, U, rounds, 0xABCD)
    lab_o, st_o = O.match(g, U, rounds, 0xABCD)
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    assert (st["rounds"], st["pairs"]) == (st_o["rounds"], st_o["pairs"])


def test_match_degenerate_inputs(gp):
    import torch
    # one vertex, no edges
    g = gg.Graph(1, np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32))
    lab, st = gp.match(gp.DeviceGraph.from_host(g), 2, 5, 1)
    assert lab.cpu().tolist() == [0] and st["pairs"] == 0
    # U below every pair: nothing is matched, one round runs
    g = gg.grid(10, 10)
    lab, st = gp.match(gp.DeviceGraph.from_host(g), 1, 5, 1)
    assert np.array_equal(lab.cpu().numpy(), np.arange(100)) and st["rounds"] == 1 and st["pairs"] == 0
    # zero rounds
    lab, st = gp.match(gp.DeviceGraph.from_host(g), 2, 0, 1)
    assert np.array_equal(lab.cpu().numpy(), np.arange(100)) and st["rounds"] == 0


@pytest.mark.parametrize("name,k", [("grid128", 4), ("rgg2e15", 16), ("rgg_weighted", 8), ("rmat12w", 8)])
def test_matching_partition_equals_oracle(gp, name, k):
    g = GRAPHS[name]()
    params = gp.default_params(coarsen=gp.COARSEN_MATCHING, coarse_min=300)
    op = O.default_params()
    op.coarsen_mode = 1
    op.coarse_min = 300
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, k, 0.03, 1, params)
    part_o, res_o = O.partition(g, k, 0.03, 1, op)
    assert res.levels == res_o.levels and res.level_n == list(res_o.level_n[: res_o.levels + 1])
    assert res.try_cut == list(res_o.try_cut[:4]) and res.best_try == res_o.best_try
    assert np.array_equal(part.cpu().numpy(), part_o)
    assert (res.cut, res.max_block_weight, res.imbalanced) == (res_o.cut, res_o.max_block_weight, res_o.imbalanced)


def test_matching_rejected_where_unsupported(gp):
    g = gg.grid(20, 20)
    dg = gp.DeviceGraph.from_host(g)
    with pytest.raises(gp.GpError):
        gp.partition_batch([dg], [2], 0.03, [1], gp.default_params(coarsen=gp.COARSEN_MATCHING))
    with pytest.raises(gp.GpError):
        gp.partition(dg, 2, 0.03, 1, gp.default_params(coarsen=7))
