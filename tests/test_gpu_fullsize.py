"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

* Random geometric graph, 2^20 vertices, average degree 12, k=16 (the default bench workload): the
  whole partition is compared element by element with the oracle (about 4 s of oracle time).
* R-MAT scale 24 (16.7M vertices, 521M CSR entries), k=16: the oracle would take minutes, so the
  result is checked through properties that hold at any size, recomputed on the host from the
  input graph: every block id in [0, k), the reported cut equals the cut of the returned partition,
  the reported block weights and balance match, degree-0 vertices are placed, and every level is
  smaller than the one before.
"""
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
