"""GPU path vs the oracle on degenerate and extreme inputs.

* stars whose hub is adjacent to 6,000-10,000 leaves: the hub path (degree above the CTA bin), movers of
  degree above 2,048 whose neighbours every block marks, and contested sets above 4,096 movers (the
  radix-sorted contest across blocks) in one small graph;
* weighted R-MAT with k = 64 (the shape of the largest configuration at test size);
* 64-bit CSR offsets (the library's int32 and int64 offset paths give identical results);
* degree-0 vertices together with general vertex weights (sequential greedy placement);
* empty and one-vertex graphs.
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


def from_edges(n, edges, weights=None, vw=None, name="edges"):
    """Symmetric CSR (rows sorted, no duplicates) from undirected edges (u, v), u != v."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(e), dtype=np.int64) if weights is None else np.asarray(weights, dtype=np.int64)
    src = np.concatenate([e[:, 0], e[:, 1]])
    dst = np.concatenate([e[:, 1], e[:, 0]])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off)
    return gg.Graph(n, off, dst.astype(np.int32), vw,
                    None if weights is None else ww.astype(np.int32), name)


def star(leaves, seed=0, path=True, chord_div=10):
    """Hub 0 with `leaves` leaves, optionally a path through the leaves, and leaves // chord_div random
    chords between leaves."""
    rng = np.random.default_rng(seed)
    n = leaves + 1
    edges = [(0, i) for i in range(1, n)] + ([(i, i + 1) for i in range(1, n - 1)] if path else [])
    chords = set()
    while len(chords) < leaves // chord_div:
        a, b = sorted(rng.integers(1, n, 2).tolist())
        if b > a + 1:
            chords.add((a, b))
    return from_edges(n, edges + sorted(chords), name="star")


def _stats_eq(a: dict, b):
    for k in ("rounds", "moves", "visits", "edges", "movers"):
        assert a[k] == getattr(b, k), (k, a[k], getattr(b, k))


def test_star_hub_big_movers_and_large_contest(gp):
    # without the path most leaves see only the hub, so about half of them contest it per sub-round
    g = star(10000, seed=1, path=False, chord_div=50)
    dg = gp.DeviceGraph.from_host(g)
    gp.profile_read(reset=True)
    gp.profile_enable(True)
    lab, st = gp.lp_cluster(dg, 97, 10, 5)
    gp.profile_enable(False)
    prof = {e["name"]: e for e in gp.profile_read(reset=True)}
    lab_o, _, st_o = O.lp_cluster(g, 97, 10, 5)
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    _stats_eq(st, st_o)
    # the paths this graph is meant to exercise were taken
    assert prof["lp_contest_large_calls"]["items"] > 0
    assert prof["lp_hub_work"]["edges"] > 0


@pytest.mark.parametrize("k", [4, 64])
def test_star_partition(gp, k):
    g = star(6000, seed=2)
    params = gp.default_params(coarse_min=300)
    op = O.default_params()
    op.coarse_min = 300
    part, res = gp.partition(gp.DeviceGraph.from_host(g), k, 0.03, 3, params)
    part_o, res_o = O.partition(g, k, 0.03, 3, op)
    assert np.array_equal(part.cpu().numpy(), part_o) and res.cut == res_o.cut


def test_weighted_rmat_k64(gp):
    g = gg.rmat(14, 16, seed=6, weighted=True)
    part, res = gp.partition(gp.DeviceGraph.from_host(g), 64, 0.03, 2)
    part_o, res_o = O.partition(g, 64, 0.03, 2)
    assert np.array_equal(part.cpu().numpy(), part_o)
    assert (res.cut, res.levels, res.max_block_weight, res.imbalanced) == (
        res_o.cut, res_o.levels, res_o.max_block_weight, res_o.imbalanced)


def test_int64_offsets_same_results(gp):
    g = gg.rmat(13, 16, seed=7, weighted=True)
    p32, r32 = gp.partition(gp.DeviceGraph.from_host(g, offsets_64=False), 8, 0.03, 4)
    p64, r64 = gp.partition(gp.DeviceGraph.from_host(g, offsets_64=True), 8, 0.03, 4)
    part_o, res_o = O.partition(g, 8, 0.03, 4)
    assert np.array_equal(p32.cpu().numpy(), part_o) and np.array_equal(p64.cpu().numpy(), part_o)
    lab32, _ = gp.lp_cluster(gp.DeviceGraph.from_host(g, offsets_64=False), 500, 10, 8)
    lab64, _ = gp.lp_cluster(gp.DeviceGraph.from_host(g, offsets_64=True), 500, 10, 8)
    assert np.array_equal(lab32.cpu().numpy(), lab64.cpu().numpy())


def test_isolated_vertices_with_vertex_weights(gp):
    base = gg.rgg(3000, 8.0, 9)
    n = base.n + 400  # 400 extra vertices without edges, some heavy
    off = np.concatenate([base.off, np.full(400, base.off[-1], dtype=base.off.dtype)])
    vw = np.random.default_rng(4).integers(1, 9, n).astype(np.int32)
    g = gg.Graph(n, off, base.adj, vw, None, "rgg+isolated")
    params = gp.default_params(coarse_min=300)
    op = O.default_params()
    op.coarse_min = 300
    part, res = gp.partition(gp.DeviceGraph.from_host(g), 6, 0.05, 5, params)
    part_o, res_o = O.partition(g, 6, 0.05, 5, op)
    assert np.array_equal(part.cpu().numpy(), part_o)
    assert (res.cut, res.n_isolated, res.max_block_weight) == (res_o.cut, res_o.n_isolated, res_o.max_block_weight)


def test_empty_and_single_vertex(gp):
    import torch
    empty = gg.Graph(0, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    de = gp.DeviceGraph.from_host(empty)
    lab, st = gp.lp_cluster(de, 1, 10, 1)
    assert lab.numel() <= 1 and st["moves"] == 0
    cg, f2c = gp.contract(de, lab[:0] if lab.numel() else lab)
    assert cg.n == 0
    cg.free()
    one = gg.Graph(1, np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32))
    part, res = gp.partition(gp.DeviceGraph.from_host(one), 1, 0.03, 1)
    assert part.cpu().numpy().tolist() == [0] and res.cut == 0 and res.n_isolated == 1


def test_choice_key_tie_takes_the_exact_order(gp):
    """With unit weights the lane-group choice first ranks candidates by the 32-bit key
    (count, top 26 bits of H(seed, v, L)) and falls back to the full order (H, then L) when two
    candidates of one vertex have equal keys. Vertex v here has exactly two neighbours whose labels
    collide in those 26 bits; its choice, and the whole clustering, must still be the oracle's."""
    seed = 4242
    smix = O.mix64(seed)
    rmix0 = O.mix64(smix ^ 0)  # round 0
    # v is active in sub-round 0 of round 0, when every neighbour still carries its own label
    v = next(x for x in range(1, 4096) if (O.mix64(rmix0 ^ x) >> 63) == 0)
    hv = O.mix64(smix ^ v)
    seen, pair = {}, None
    for L in range(v + 1, v + (1 << 17)):
        key = O.mix64(hv ^ L) >> 38
        if key in seen:
            pair = (seen[key], L)
            break
        seen[key] = L
    assert pair is not None
    l1, l2 = pair
    assert O.mix64(hv ^ l1) != O.mix64(hv ^ l2)  # equal keys, different full hashes
    g = from_edges(l2 + 1, [(v, l1), (v, l2)], name="key_tie")
    dg = gp.DeviceGraph.from_host(g)
    lab, st = gp.lp_cluster(dg, 8, 4, seed)
    lab_o, _, st_o = O.lp_cluster(g, 8, 4, seed)
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    _stats_eq(st, st_o)
