"""Learned edge scorer on the GPU vs the FP64 oracle; learned-mode LP and partition vs the oracle.

* features: GPU float features vs oracle FP64 features;
* inference: |s_gpu - s_fp64| <= 1e-2 with the same BF16 weights (BF16 tensor-core path);
* q = round-half-even(s * 2^15) of the GPU's own float scores;
* gradients: GPU FP32 gradients vs oracle FP64 gradients within 2e-2 relative or 1e-3 absolute;
* learned-mode partition: bit-exact with the oracle given the GPU's quantised scores per level
  (the oracle takes q as input, so LP parity stays exact);
* a trained scorer is compared with plain LP at the same seeds (the gain is reported, not assumed).
"""
import math

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


def _weights(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return (rng.normal(0, scale, (32, 8)), rng.normal(0, 0.1, 32), rng.normal(0, scale, 32), float(rng.normal(0, 0.1)))


def _vw_graph():
    g = gg.rgg(3000, 9.0, 5)
    g.vw = np.random.default_rng(2).integers(1, 5, g.n).astype(np.int32)
    return g


GRAPHS = {"grid": lambda: gg.grid(33, 47), "rmat12w": lambda: gg.rmat(12, 16, seed=4, weighted=True),
          "rgg_vw": _vw_graph}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_features_match_oracle(gp, name):
    g = GRAPHS[name]()
    dg = gp.DeviceGraph.from_host(g)
    f = gp.edge_features(dg, 3).cpu().numpy().astype(np.float64)
    fo = O.edge_features(g, 3)
    assert f.shape == fo.shape
    assert np.allclose(f, fo, rtol=2e-6, atol=2e-6), np.abs(f - fo).max()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_scores_within_1e2_of_fp64(gp, name):
    g = GRAPHS[name]()
    dg = gp.DeviceGraph.from_host(g)
    w1, b1, w2, b2 = _weights(7)
    mlp = gp.mlp_pack(w1, b1, w2, b2)
    s, q = gp.mlp_score(dg, 1, mlp)
    s = s.cpu().numpy()
    q = q.cpu().numpy()
    bw1, bb1, bw2, bb2 = gp.mlp_unpack(mlp)  # the BF16 weights the GPU used, exactly
    s64 = O.mlp_forward(O.edge_features(g, 1), bw1, bb1, bw2, bb2)
    assert np.abs(s.astype(np.float64) - s64).max() <= 1e-2
    # q is the GPU float score times 2^15 rounded half to even
    assert np.array_equal(q, np.rint(s.astype(np.float32) * np.float32(32768.0)).astype(np.int32))
    # symmetric: entry (v,u) and (u,v) score the same
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    order = np.lexsort((g.adj, src))
    rev = np.lexsort((src, g.adj))
    assert np.array_equal(q[order], q[rev])


def test_gradients_match_fp64(gp):
    import torch
    g = GRAPHS["rmat12w"]()
    dg = gp.DeviceGraph.from_host(g)
    feat = gp.edge_features(dg, 0)
    rng = np.random.default_rng(3)
    y = (rng.random(g.m_dir) < 0.4).astype(np.float32)
    w1, b1, w2, b2 = _weights(11, 0.3)
    mlp = gp.mlp_pack(w1, b1, w2, b2)
    loss, grad = gp.mlp_grad(feat, torch.from_numpy(y).cuda(), mlp)
    bw1, bb1, bw2, bb2 = gp.mlp_unpack(mlp)
    loss64, gw1, gb1, gw2, gb2 = O.mlp_loss_grad(feat.cpu().numpy().astype(np.float64), y.astype(np.float64),
                                                 bw1, bb1, bw2, bb2)
    want = np.concatenate([gw1.reshape(-1), gb1, gw2, [gb2]])
    got = grad.astype(np.float64)
    ok = (np.abs(got - want) <= 1e-3) | (np.abs(got - want) <= 2e-2 * np.abs(want))
    assert ok.all(), np.abs(got - want).max()
    assert abs(loss - loss64) <= 1e-4 * max(1.0, abs(loss64))


def test_training_reduces_loss(gp):
    import torch
    g = gg.rmat(11, 16, seed=9)
    dg = gp.DeviceGraph.from_host(g)
    feat = gp.edge_features(dg, 0)
    part, _ = gp.partition(dg, 4, 0.03, 1)
    p = part.cpu().numpy()
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    y = torch.from_numpy((p[src] == p[g.adj]).astype(np.float32)).cuda()
    mlp = gp.mlp_pack(*_weights(5, 0.2))
    losses = gp.mlp_train(feat, y, mlp, 150, 2e-2)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < losses[0]


def _learned_levels(gp, g, mlp, k, eps, seed, coarse_min):
    """q of every coarsening level, rebuilt through the C ABI exactly as the learned partition
    coarsens (the test graph has no degree-0 vertices)."""
    import torch
    W = int(O.vertex_weights(g).sum())
    lmax = O.lmax(W, k, eps)
    T = max(coarse_min, 64 * k)
    dg = gp.DeviceGraph.from_host(g)
    qs, cur = [], g
    holders = []
    level = 0
    while cur.n > T and level < 64:
        _, q = gp.mlp_score(dg, level, mlp)
        qs.append(q.cpu().numpy())
        c = O.vertex_weights(cur)
        U = max(int(c.max()), lmax // 14)
        lab, _ = gp.lp_cluster(dg, U, 10, O.hash3(seed, level, 1), q=q)
        cg, _ = gp.contract(dg, lab)
        holders.append(cg)
        nxt = cg.to_host()
        dg = gp.DeviceGraph(nxt.n, torch.from_numpy(nxt.off).cuda(), torch.from_numpy(nxt.adj).cuda(),
                            torch.from_numpy(nxt.vw).cuda(), torch.from_numpy(nxt.ew).cuda())
        level += 1
        stalled = 100 * nxt.n > 95 * cur.n
        cur = nxt
        if stalled:
            break
    return qs


@pytest.mark.parametrize("name,k", [("rgg14", 8), ("grid", 4)])
def test_learned_partition_matches_oracle(gp, name, k):
    g = gg.rgg(1 << 14, 12.0, 3) if name == "rgg14" else gg.grid(120, 90)
    assert (np.diff(g.off) > 0).all()
    w1, b1, w2, b2 = _weights(21, 0.4)
    mlp = gp.mlp_pack(w1, b1, w2, b2)
    params = gp.default_params(mode=gp.MODE_LEARNED, coarse_min=500)
    params.mlp = mlp.data_ptr()
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, k, 0.03, 5, params)
    qs = _learned_levels(gp, g, mlp, k, 0.03, 5, 500)
    op = O.default_params()
    op.coarse_min = 500
    part_o, res_o = O.partition(g, k, 0.03, 5, op, q_levels=qs)
    assert res.levels == res_o.levels == len(qs)
    assert np.array_equal(part.cpu().numpy(), part_o)
    assert res.cut == res_o.cut and res.learned_cut == res.cut


def test_best_of_reports_both_cuts(gp):
    g = gg.rmat(12, 16, seed=31)
    dg = gp.DeviceGraph.from_host(g)
    mlp = gp.mlp_pack(*_weights(3, 0.4))
    pl = gp.default_params()
    _, rp = gp.partition(dg, 8, 0.03, 2, pl)
    ll = gp.default_params(mode=gp.MODE_LEARNED)
    ll.mlp = mlp.data_ptr()
    _, rl = gp.partition(dg, 8, 0.03, 2, ll)
    bo = gp.default_params(mode=gp.MODE_BEST_OF)
    bo.mlp = mlp.data_ptr()
    part, rb = gp.partition(dg, 8, 0.03, 2, bo)
    assert rb.plain_cut == rp.cut and rb.learned_cut == rl.cut
    use_learned = rl.imbalanced <= rp.imbalanced and rl.cut < rp.cut
    assert rb.cut == (rl.cut if use_learned else rp.cut)


def _uncut_labels(g, part):
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    return (part[src] == part[g.adj]).astype(np.float32)


def _train_balanced(gp, graphs, k):
    """The scorer trained on which edges plain partitions leave uncut, classes balanced (every cut edge
    and as many uncut edges, drawn with a fixed seed)."""
    import torch
    feats, ys = [], []
    rng = np.random.default_rng(1)
    for g in graphs:
        dg = gp.DeviceGraph.from_host(g)
        part, _ = gp.partition(dg, k, 0.03, 1)
        y = _uncut_labels(g, part.cpu().numpy()) > 0
        pos, neg = np.flatnonzero(y), np.flatnonzero(~y)
        keep = np.sort(np.concatenate([neg, rng.choice(pos, min(len(pos), len(neg)), replace=False)]))
        feats.append(gp.edge_features(dg, 0)[torch.from_numpy(keep).cuda()].contiguous())
        ys.append(torch.from_numpy(y[keep].astype(np.float32)).cuda())
    mlp = gp.mlp_pack(*_weights(1, 0.2))
    losses = gp.mlp_train(torch.cat(feats).contiguous(), torch.cat(ys), mlp, 300, 1e-2)
    return mlp, losses


def test_trained_scorer_gains_on_power_law_graphs(gp):
    """What the trained network gains over the method without it: trained on R-MAT scale-14 graphs of
    other seeds, the learned partition of a held-out R-MAT scale-17 graph has a lower cut than the plain
    one at the same seed (geometric mean over seeds 1-5 below 0.99, at least four of five not worse;
    measured on R-MAT scale 24: 0.925 over seeds 1-10). BEST_OF never loses to plain."""
    mlp, losses = _train_balanced(gp, [gg.rmat(14, 16, seed=s) for s in (101, 102)], 16)
    assert losses[-1] < losses[0]
    g = gg.rmat(17, 16, seed=7)
    dg = gp.DeviceGraph.from_host(g)
    ratios = []
    for seed in range(1, 6):
        _, rp = gp.partition(dg, 16, 0.03, seed)
        bo = gp.default_params(mode=gp.MODE_BEST_OF)
        bo.mlp = mlp.data_ptr()
        _, rb = gp.partition(dg, 16, 0.03, seed, bo)
        assert rb.plain_cut == rp.cut and rb.cut <= rp.cut
        ratios.append(rb.learned_cut / rp.cut)
    gmean = math.exp(np.mean(np.log(ratios)))
    print(f"learned/plain cut ratios {[round(r, 4) for r in ratios]}, geometric mean {gmean:.4f}")
    assert gmean < 0.99
    assert sum(r <= 1.0 for r in ratios) >= 4
