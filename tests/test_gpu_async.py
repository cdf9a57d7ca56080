"""The paper's asynchronous LP on the GPU (gp_lp_cluster_async, Section IV-A), the comparator for the
deterministic Jacobi rounds.

* On one warp the order is the sequential one of Section III-A: labels and counters must equal the
  oracle's (oracle.lp_async) element by element.
* On the whole GPU the result depends on the interleaving of the warps, so it is checked through what
  must hold in any interleaving: every label is a vertex id, no cluster exceeds U (the compare-and-swap
  reservation), and a partition built on it is consistent (cut and block weights recomputed on the
  host, balance flag).
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
    return m


def _weighted_rgg(n, seed):
    g = gg.rgg(n, 9.0, seed)
    rng = np.random.default_rng(seed)
    g.vw = rng.integers(1, 4, g.n).astype(np.int32)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    lo, hi = np.minimum(src, g.adj), np.maximum(src, g.adj)
    g.ew = (1 + (lo * 31 + hi * 17) % 5).astype(np.int32)
    return g


GRAPHS = {
    "grid64": lambda: gg.grid(64, 64),
    "rgg2e13": lambda: gg.rgg(1 << 13, 12.0, 2),
    "rgg_weighted": lambda: _weighted_rgg(6000, 3),
    "rmat9": lambda: gg.rmat(9, 4, seed=7),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("U", [3, 40])
def test_single_warp_equals_sequential_oracle(gp, name, U):
    g = GRAPHS[name]()
    U = max(U, int(O.vertex_weights(g).max()))
    dg = gp.DeviceGraph.from_host(g)
    lab, st = gp.lp_cluster_async(dg, U, 10, 0x51, single_warp=True)
    lab_o, lw_o, st_o = O.lp_cluster_async(g, U, 10, 0x51)
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    assert (st["rounds"], st["moves"], st["visits"], st["edges"]) == (st_o.rounds, st_o.moves, st_o.visits, st_o.edges)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_parallel_keeps_the_size_bound(gp, name):
    g = GRAPHS[name]()
    c = O.vertex_weights(g)
    U = max(30, int(c.max()))
    dg = gp.DeviceGraph.from_host(g)
    lab, st = gp.lp_cluster_async(dg, U, 10, 3)
    lab = lab.cpu().numpy()
    assert lab.min() >= 0 and lab.max() < g.n
    w = np.bincount(lab, weights=c, minlength=g.n)
    assert w.max() <= U
    assert st["moves"] > 0


@pytest.mark.parametrize("name,k", [("rgg2e13", 8), ("rgg_weighted", 4), ("grid64", 2)])
def test_async_partition_is_consistent(gp, name, k):
    g = GRAPHS[name]()
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, k, 0.03, 1, gp.default_params(lp_async=1, coarse_min=300))
    p = part.cpu().numpy()
    assert p.min() >= 0 and p.max() < k
    cut, bw = O.cut(g, p, k)
    assert res.cut == cut and res.max_block_weight == bw.max()
    assert res.imbalanced == int(bw.max() > res.lmax)


def test_async_rejects_wide_label_sets(gp):
    g = gg.rmat(12, 16, seed=1)  # degrees above 256
    with pytest.raises(gp.GpError) as ei:
        gp.lp_cluster_async(gp.DeviceGraph.from_host(g), 50, 10, 1)
    assert ei.value.status == gp.GP_ERR_UNSUPPORTED
