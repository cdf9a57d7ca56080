"""GPU multi-try k-way local search (gp_mls) and MLS-refined partitions against the oracle, element by
element: the partition after every global and local iteration's PerformMoves and ApplyMoves, the
gain, moves, searches and local iterations, and the whole partition with mls_global_iters = 3.

Start partitions are LP-refined partitions (the state MLS runs on in the multilevel scheme) and, for
more moves, random or perturbed ones; graphs are meshes, weighted meshes and R-MAT graphs whose hubs
lie above the degree bound."""
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
    "grid96": lambda: gg.grid(96, 96),
    "rgg2e14": lambda: gg.rgg(1 << 14, 10.0, 3),
    "rgg_weighted": lambda: _weighted_rgg(12000, 4),
    "rmat11": lambda: gg.rmat(11, 8, seed=5),
}


def _start(g, k, how, seed):
    if how == "lp":
        part, _ = O.partition(g, k, 0.03, seed)
        return part
    rng = np.random.default_rng(seed)
    part, _ = O.partition(g, k, 0.03, seed)
    flip = rng.random(g.n) < 0.05  # perturbed: 5% of the vertices in a random block
    part = part.copy()
    part[flip] = rng.integers(0, k, int(flip.sum()))
    return part.astype(np.int32)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("k,how", [(2, "lp"), (8, "lp"), (16, "perturbed"), (64, "perturbed")])
def test_mls_equals_oracle(gp, name, k, how):
    import torch
    g = GRAPHS[name]()
    part0 = _start(g, k, how, 3)
    c = O.vertex_weights(g)
    lmax = max(O.lmax(int(c.sum()), k, 0.03), int(np.bincount(part0, weights=c, minlength=k).max()))
    dg = gp.DeviceGraph.from_host(g)
    out, st = gp.mls(dg, torch.from_numpy(part0).cuda(), k, lmax, 0x77)
    out_o, st_o = O.mls(g, part0, k, lmax, 0x77)
    assert np.array_equal(out.cpu().numpy(), out_o)
    assert st == st_o


@pytest.mark.parametrize("over", [dict(max_moves=1, fruitless=1), dict(max_moves=8, fruitless=2, queue_cap=4),
                                  dict(max_degree=6), dict(global_iters=1, alpha_pct=50), dict(max_local=1)])
def test_mls_parameters_equal_oracle(gp, over):
    import torch
    g = GRAPHS["rgg_weighted"]()
    k = 8
    part0 = _start(g, k, "perturbed", 9)
    c = O.vertex_weights(g)
    lmax = max(O.lmax(int(c.sum()), k, 0.03), int(np.bincount(part0, weights=c, minlength=k).max()))
    p = gp.mls_default_params(**over)
    po = O.mls_default_params()
    for a, v in over.items():
        setattr(po, a, v)
    dg = gp.DeviceGraph.from_host(g)
    out, st = gp.mls(dg, torch.from_numpy(part0).cuda(), k, lmax, 5, p)
    out_o, st_o = O.mls(g, part0, k, lmax, 5, po)
    assert np.array_equal(out.cpu().numpy(), out_o) and st == st_o


@pytest.mark.parametrize("name,k", [("rgg2e14", 8), ("rgg_weighted", 4), ("rmat11", 16)])
def test_mls_partition_equals_oracle(gp, name, k):
    g = GRAPHS[name]()
    params = gp.default_params(mls_global_iters=3, coarse_min=300)
    op = O.default_params()
    op.mls = 3
    op.coarse_min = 300
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, k, 0.03, 1, params)
    part_o, res_o = O.partition(g, k, 0.03, 1, op)
    assert np.array_equal(part.cpu().numpy(), part_o)
    assert (res.cut, res.max_block_weight, res.imbalanced) == (res_o.cut, res_o.max_block_weight, res_o.imbalanced)
    # and MLS does not make the partition worse than LP refinement alone at the same seed
    _, plain = gp.partition(dg, k, 0.03, 1, gp.default_params(coarse_min=300))
    assert res.cut <= plain.cut


def test_mls_rejects_unsupported(gp):
    import torch
    g = gg.grid(20, 20)
    dg = gp.DeviceGraph.from_host(g)
    part = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(gp.GpError):
        gp.mls(dg, part, 300, 10**6, 1)  # k > 256
    with pytest.raises(gp.GpError):
        gp.mls(dg, part, 2, 10**6, 1, gp.mls_default_params(max_moves=65))
