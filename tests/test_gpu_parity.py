"""GPU path vs the CPU oracle, element by element (labels, coarse CSR, partitions, cuts, stats).

All integer results must be bit-identical. Inputs are seeded synthetic graphs of the paper's
workload families (grid/mesh, random geometric, R-MAT power law, weighted R-MAT)."""
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


def _graphs():
    g_vw = gg.rgg(3000, 9.0, 5)
    g_vw.vw = np.random.default_rng(2).integers(1, 5, g_vw.n).astype(np.int32)
    return {
        "grid256": gg.grid(256, 256),
        "grid_ragged": gg.grid(37, 53),
        "rgg15": gg.rgg(1 << 15, 12.0, 1),
        "rmat13": gg.rmat(13, 16, seed=3),
        "rmat12w": gg.rmat(12, 16, seed=4, weighted=True),
        "rgg_vw": g_vw,
    }


GRAPHS = _graphs()


def _stats_eq(a: dict, b):
    for k in ("rounds", "moves", "visits", "edges", "movers"):
        assert a[k] == getattr(b, k), (k, a[k], getattr(b, k))


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("sched", [(0, 0), (32, 32), (256, 2048)])
def test_lp_cluster_matches_oracle(gp, name, sched):
    g = GRAPHS[name]
    gp.lp_set_schedule(*sched)
    try:
        dg = gp.DeviceGraph.from_host(g)
        c = O.vertex_weights(g)
        U = int(max(c.max(), 40))
        seed = 0xC0FFEE
        lab, st = gp.lp_cluster(dg, U, 10, seed)
        lab_o, lw_o, st_o = O.lp_cluster(g, U, 10, seed)
        assert np.array_equal(lab.cpu().numpy(), lab_o)
        _stats_eq(st, st_o)
    finally:
        gp.lp_set_schedule(0, 0)


@pytest.mark.parametrize("name", ["rgg15", "rmat13", "rmat12w"])
def test_lp_cluster_learned_scores_match_oracle(gp, name):
    import torch
    g = GRAPHS[name]
    rng = np.random.default_rng(7)
    # symmetric per-edge scores in [0, 2^15]
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    key = np.minimum(src, g.adj).astype(np.int64) * g.n + np.maximum(src, g.adj)
    q = (np.vectorize(lambda x: O.mix64(int(x)) & 0x7FFF, otypes=[np.int64])(key)).astype(np.int32)
    dg = gp.DeviceGraph.from_host(g)
    lab, st = gp.lp_cluster(dg, 60, 10, 99, q=torch.from_numpy(q).cuda())
    lab_o, _, st_o = O.lp_cluster(g, 60, 10, 99, q=q)
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    _stats_eq(st, st_o)


@pytest.mark.parametrize("name", ["rgg15", "rmat13"])
@pytest.mark.parametrize("bits", [15, 20])
def test_lp_cluster_score_ranges_match_oracle(gp, name, bits):
    """Scores up to 2^15 (the scorer's range) take the packed-key choice with unit weights; wider
    scores take the general reduction. Both must equal the oracle."""
    import torch
    g = GRAPHS[name]
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    key = np.minimum(src, g.adj).astype(np.int64) * g.n + np.maximum(src, g.adj)
    mask = (1 << bits) - 1
    q = (np.vectorize(lambda x: O.mix64(int(x) ^ 0x5A5A) & mask, otypes=[np.int64])(key)).astype(np.int32)
    if bits == 15:
        q[::7] = 1 << 15  # the top of the scorer's range
    dg = gp.DeviceGraph.from_host(g)
    lab, st = gp.lp_cluster(dg, 60, 10, 17, q=torch.from_numpy(q).cuda())
    lab_o, _, st_o = O.lp_cluster(g, 60, 10, 17, q=q)
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    _stats_eq(st, st_o)


@pytest.mark.parametrize("name", ["grid256", "rgg15", "rmat13", "rmat12w", "rgg_vw"])
@pytest.mark.parametrize("k", [2, 16])
def test_lp_refine_matches_oracle(gp, name, k):
    import torch
    g = GRAPHS[name]
    rng = np.random.default_rng(k)
    part = rng.integers(0, k, g.n).astype(np.int32)
    c = O.vertex_weights(g)
    lm = O.lmax(int(c.sum()), k, 0.03)
    dg = gp.DeviceGraph.from_host(g)
    p, bw, st = gp.lp_refine(dg, torch.from_numpy(part).cuda(), k, lm, 25, 1234)
    p_o, bw_o, st_o = O.lp_refine(g, part, k, lm, 25, 1234)
    assert np.array_equal(p.cpu().numpy(), p_o)
    assert np.array_equal(bw.cpu().numpy(), bw_o)
    _stats_eq(st, st_o)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_contract_matches_oracle(gp, name):
    import torch
    g = GRAPHS[name]
    lab_o, _, _ = O.lp_cluster(g, 30, 10, 5)
    dg = gp.DeviceGraph.from_host(g)
    cg, f2c = gp.contract(dg, torch.from_numpy(lab_o).cuda())
    h = cg.to_host()
    co, f2c_o = O.contract(g, lab_o)
    assert h.n == co.n
    assert np.array_equal(f2c.cpu().numpy(), f2c_o)
    assert np.array_equal(h.off, co.off)
    assert np.array_equal(h.adj, co.adj)
    assert np.array_equal(h.vw, co.vw)
    assert np.array_equal(h.ew, co.ew)
    cg.free()


def test_contract_arbitrary_labels(gp):
    import torch
    g = GRAPHS["rmat13"]
    rng = np.random.default_rng(11)
    lab = rng.integers(0, 50, g.n).astype(np.int32)  # few huge clusters: the large-row path
    dg = gp.DeviceGraph.from_host(g)
    cg, f2c = gp.contract(dg, torch.from_numpy(lab).cuda())
    h = cg.to_host()
    co, f2c_o = O.contract(g, lab)
    for a, b in [(h.off, co.off), (h.adj, co.adj), (h.vw, co.vw), (h.ew, co.ew), (f2c.cpu().numpy(), f2c_o)]:
        assert np.array_equal(a, b)
    cg.free()


PARTS = [("grid256", 2), ("grid_ragged", 3), ("rgg15", 16), ("rmat13", 16), ("rmat12w", 8), ("rgg_vw", 4)]


@pytest.mark.parametrize("name,k", PARTS)
def test_partition_matches_oracle(gp, name, k):
    g = GRAPHS[name]
    params = gp.default_params()
    oparams = O.default_params()
    if g.n < 20000:
        params.coarse_min = oparams.coarse_min = 300
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, k, 0.03, 1, params)
    part_o, res_o = O.partition(g, k, 0.03, 1, oparams)
    assert res.levels == res_o.levels
    assert res.level_n == list(res_o.level_n[: res_o.levels + 1])
    assert res.level_m == list(res_o.level_m[: res_o.levels + 1])
    assert res.try_cut == list(res_o.try_cut[:4])
    assert res.best_try == res_o.best_try
    assert np.array_equal(part.cpu().numpy(), part_o)
    assert (res.cut, res.max_block_weight, res.lmax, res.imbalanced, res.n_isolated) == (
        res_o.cut, res_o.max_block_weight, res_o.lmax, res_o.imbalanced, res_o.n_isolated)
    assert res.lp_edges == res_o.lp_edges


def test_partition_edge_cases(gp):
    import torch
    # no edges at all: every vertex is degree-0 and goes to the lightest block
    n = 10
    g = gg.Graph(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, 3, 0.0, 1)
    part_o, res_o = O.partition(g, 3, 0.0, 1)
    assert np.array_equal(part.cpu().numpy(), part_o) and res.cut == 0
    # k = 1 and k = n on a small grid
    g = gg.grid(4, 5)
    dg = gp.DeviceGraph.from_host(g)
    for k in (1, g.n):
        part, res = gp.partition(dg, k, 0.03, 2)
        part_o, res_o = O.partition(g, k, 0.03, 2)
        assert np.array_equal(part.cpu().numpy(), part_o) and res.cut == res_o.cut
    # invalid k is an error, not a crash
    with pytest.raises(gp.GpError):
        gp.partition(dg, 0, 0.03, 1)
    with pytest.raises(gp.GpError):
        gp.partition(dg, g.n + 1, 0.03, 1)


def test_partition_host_buffers(gp):
    g = GRAPHS["rgg15"]
    hg = gp.HostGraph(g)
    part, res = gp.partition_host(hg, 16, 0.03, 1)
    part_o, res_o = O.partition(g, 16, 0.03, 1)
    assert np.array_equal(part, part_o) and res.cut == res_o.cut


def test_validate_rejects_bad_graphs(gp):
    g = gg.grid(8, 8)
    assert gp.validate(gp.DeviceGraph.from_host(g)) == 0
    bad = gg.Graph(g.n, g.off.copy(), g.adj.copy())
    bad.adj[3] = bad.adj[2]  # duplicate / unsorted entry
    assert gp.validate(gp.DeviceGraph.from_host(bad)) == gp.GP_ERR_BAD_GRAPH
    asym = gg.Graph(g.n, g.off.copy(), g.adj.copy(), None, np.ones(g.m_dir, dtype=np.int32))
    asym.ew[0] = 2
    assert gp.validate(gp.DeviceGraph.from_host(asym)) == gp.GP_ERR_BAD_GRAPH


def test_determinism_repeated_runs(gp):
    g = GRAPHS["rmat13"]
    dg = gp.DeviceGraph.from_host(g)
    outs = [gp.partition(dg, 16, 0.03, 9)[0].cpu().numpy() for _ in range(3)]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


# ---- the hub path (vertices above deg_cta, several CTAs each). Three forms must give the oracle's
# result: tables re-accumulated every sub-round in batches (a small batch size splits the hubs of one
# sub-round into many batches, each with its own table pass); tables kept across sub-rounds and updated
# by the moves (the default); kept tables that go stale at their first new label and are accumulated
# again at the hub's next activation.
HUB_CASES = [("rmat13", 32, 32, 4096), ("rmat13", 0, 0, 4096), ("rmat12w", 32, 64, 8192),
             ("rmat14", 32, 32, 16384)]
HUB_FORMS = {"batches": (-1, 0), "kept": (0, 0), "kept_stale": (0, 1)}


@pytest.mark.parametrize("form", list(HUB_FORMS))
@pytest.mark.parametrize("name,dw,dc,slots", HUB_CASES)
def test_lp_cluster_hub_forms_match_oracle(gp, name, dw, dc, slots, form):
    g = GRAPHS[name] if name in GRAPHS else gg.rmat(14, 16, seed=8)
    gp.lp_set_schedule(dw, dc)
    gp.lp_set_tiles(slots, 0)
    gp.lp_set_hub_keep(*HUB_FORMS[form])
    try:
        dg = gp.DeviceGraph.from_host(g)
        gp.profile_read(reset=True)
        gp.profile_enable(True)
        lab, st = gp.lp_cluster(dg, 200, 10, 0xBEEF)
        gp.profile_enable(False)
        prof = {e["name"]: e for e in gp.profile_read(reset=True)}
        lab_o, _, st_o = O.lp_cluster(g, 200, 10, 0xBEEF)
        assert np.array_equal(lab.cpu().numpy(), lab_o)
        _stats_eq(st, st_o)
        work, built = prof["lp_hub_work"], prof["lp_hub_built"]
        assert work["items"] > 0
        if form == "batches":
            # the hub tables of a sub-round with every vertex active are several batches' worth
            d = np.diff(g.off)
            hubs = d[d > (dc or 1024)]
            assert ((2 * hubs + 63) // 64 * 64).sum() > 4 * slots
            assert built["edges"] == work["edges"]  # every active hub accumulated every sub-round
        elif form == "kept":
            assert built["edges"] < work["edges"]  # some hub sub-rounds followed the moves
        else:
            assert built["items"] > 0  # tables went stale and were accumulated again
    finally:
        gp.lp_set_schedule(0, 0)
        gp.lp_set_tiles(0, 0)
        gp.lp_set_hub_keep(0, 0)


@pytest.mark.parametrize("form", list(HUB_FORMS))
@pytest.mark.parametrize("name", ["rmat13", "rmat12w"])
def test_lp_cluster_scored_hub_forms_match_oracle(gp, name, form):
    """Runs with scores (symmetric, up to 2^20 so that a label's score sum can pass 2^32 only in 64 bits
    on larger graphs) through every hub form: kept tables move the score sums with the weights."""
    import torch
    g = GRAPHS[name]
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    key = np.minimum(src, g.adj).astype(np.int64) * g.n + np.maximum(src, g.adj)
    q = (np.vectorize(lambda x: O.mix64(int(x) ^ 0x3C3C) & 0xFFFFF, otypes=[np.int64])(key)).astype(np.int32)
    dg = gp.DeviceGraph.from_host(g)
    gp.lp_set_schedule(32, 32)
    gp.lp_set_tiles(4096, 0)
    gp.lp_set_hub_keep(*HUB_FORMS[form])
    try:
        lab, st = gp.lp_cluster(dg, 150, 10, 23, q=torch.from_numpy(q).cuda())
    finally:
        gp.lp_set_schedule(0, 0)
        gp.lp_set_tiles(0, 0)
        gp.lp_set_hub_keep(0, 0)
    lab_o, _, st_o = O.lp_cluster(g, 150, 10, 23, q=q)
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    _stats_eq(st, st_o)


@pytest.mark.parametrize("form", ["batches", "kept_stale"])
@pytest.mark.parametrize("name,k", [("rmat13", 16), ("rmat12w", 8)])
def test_lp_refine_and_partition_hub_forms_match_oracle(gp, name, k, form):
    import torch
    g = GRAPHS[name]
    c = O.vertex_weights(g)
    lm = O.lmax(int(c.sum()), k, 0.03)
    part = np.random.default_rng(3).integers(0, k, g.n).astype(np.int32)
    dg = gp.DeviceGraph.from_host(g)
    keep, pct = HUB_FORMS[form]
    params = gp.default_params(deg_warp=32, deg_cta=32, hub_batch_slots=4096, coarse_min=300, hub_keep_slots=keep)
    oparams = O.default_params()
    oparams.coarse_min = 300
    gp.lp_set_schedule(32, 32)
    gp.lp_set_tiles(4096, 0)
    gp.lp_set_hub_keep(keep, pct)
    try:
        p, bw, st = gp.lp_refine(dg, torch.from_numpy(part).cuda(), k, lm, 25, 77)
        pp, res = gp.partition(dg, k, 0.03, 5, params)
    finally:
        gp.lp_set_schedule(0, 0)
        gp.lp_set_tiles(0, 0)
        gp.lp_set_hub_keep(0, 0)
    p_o, bw_o, st_o = O.lp_refine(g, part, k, lm, 25, 77)
    assert np.array_equal(p.cpu().numpy(), p_o) and np.array_equal(bw.cpu().numpy(), bw_o)
    _stats_eq(st, st_o)
    pp_o, res_o = O.partition(g, k, 0.03, 5, oparams)
    assert np.array_equal(pp.cpu().numpy(), pp_o) and res.cut == res_o.cut


@pytest.mark.parametrize("vpb", [16, 32, 256, 4096])
def test_tile_sizes_never_change_results(gp, vpb):
    g = GRAPHS["rgg15"]
    dg = gp.DeviceGraph.from_host(g)
    ref, st_ref = gp.lp_cluster(dg, 50, 10, 31)
    gp.lp_set_tiles(0, vpb)
    try:
        lab, st = gp.lp_cluster(dg, 50, 10, 31)
    finally:
        gp.lp_set_tiles(0, 0)
    assert np.array_equal(lab.cpu().numpy(), ref.cpu().numpy()) and st == st_ref
    part, res = gp.partition(dg, 16, 0.03, 1, gp.default_params(verts_per_block=vpb))
    part_o, res_o = O.partition(g, 16, 0.03, 1)
    assert np.array_equal(part.cpu().numpy(), part_o)


def test_autotune_picks_valid_tiles_and_keeps_results(gp):
    g = GRAPHS["rmat13"]
    dg = gp.DeviceGraph.from_host(g)
    params, ms = gp.autotune(dg)
    assert ms > 0
    assert params.verts_per_block in (32, 64, 128, 256)
    assert params.hub_batch_slots in (0, 1 << 22, 1 << 24, 1 << 26)
    part, res = gp.partition(dg, 16, 0.03, 1, params)
    part_o, res_o = O.partition(g, 16, 0.03, 1)
    assert np.array_equal(part.cpu().numpy(), part_o)


@pytest.mark.parametrize("tries", [1, 7, 8, 16])
@pytest.mark.parametrize("name,k", [("rgg15", 16), ("rmat12w", 8)])
def test_partition_ip_tries_match_oracle(gp, tries, name, k):
    """More initial-partitioning tries run as more problems of the same launches (Section IV-B: tries in
    parallel); every try's cut and the try kept equal the oracle's."""
    g = GRAPHS[name]
    params = gp.default_params(ip_tries=tries)
    oparams = O.default_params()
    oparams.ip_tries = tries
    if g.n < 20000:
        params.coarse_min = oparams.coarse_min = 300
    dg = gp.DeviceGraph.from_host(g)
    part, res = gp.partition(dg, k, 0.03, 3, params)
    part_o, res_o = O.partition(g, k, 0.03, 3, oparams)
    assert res.try_cut == list(res_o.try_cut[:tries])
    assert res.try_imbalanced == list(res_o.try_imbalanced[:tries])
    assert res.best_try == res_o.best_try
    assert np.array_equal(part.cpu().numpy(), part_o) and res.cut == res_o.cut
