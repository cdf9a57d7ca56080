"""Pins of the CPU oracle against facts fixed outside the oracle itself.

What pins each oracle function:

* ``mix64`` / ``hash3``  -- the published SplitMix64 output sequence for seed 0.
* ``lmax``               -- the closed form of Section II-A on exact values.
* ``lp``                 -- three hand-traced runs (tests/golden/lp_hand.json), a brute-force
                            check of the first sub-round's decisions, and invariants (label
                            weights equal the vertex-weight sums, no cluster exceeds U).
* ``contract``           -- a brute-force dictionary quotient graph, the totals of Section III-A,
                            and the cut/balance preservation claim of Section III-A.
* ``cut``                -- sum of crossing weights over an explicit edge list.
* ``bisect``/``repair``  -- hand-traced cases (tests/golden/ip_hand.json).
* ``partition``          -- brute-force optimum on tiny graphs (lower bound), balance, the
                            closed-form water-filling of the degree-0 vertex rule; its driver (stop
                            rule, seeds, try choice, projection) by tests/test_oracle_driver.py.
* ``mlp_*``              -- a closed-form forward case and central finite differences.
* ``edge_features``      -- values worked by hand on a small graph.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _graph(case):
    ew = None if case.get("ew") is None else np.array(case["ew"], dtype=np.int64)
    vw = None if case.get("vw") is None else np.array(case["vw"], dtype=np.int64)
    return gg.Graph(case["n"], np.array(case["off"], dtype=np.int64), np.array(case["adj"], dtype=np.int32), vw, ew)


def _edges(g):
    out = []
    for v in range(g.n):
        for e in range(g.off[v], g.off[v + 1]):
            u = int(g.adj[e])
            if v < u:
                out.append((v, u, 1 if g.ew is None else int(g.ew[e])))
    return out


# ------------------------------------------------------------------------------------- hash
def test_mix64_published_splitmix64_sequence():
    # SplitMix64 (Steele, Lea & Flood 2014) from state 0: state += golden gamma, output = mix(state).
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
                0x1B39896A51A8749B]
    state = 0
    for want in expected:
        state = (state + 0x9E3779B97F4A7C15) % (1 << 64)
        assert O.mix64(state) == want


def test_hash3_is_nested_mix():
    for a, b, c in [(0, 0, 0), (1, 2, 3), (2**63 + 5, 17, 2**40)]:
        assert O.hash3(a, b, c) == O.mix64(O.mix64(O.mix64(a) ^ b) ^ c)


# ------------------------------------------------------------------------------------- Lmax
@pytest.mark.parametrize("W,k,eps,want", [
    (65536, 2, 0.03, 33751),      # 1.03 * 32768 = 33751.04
    (100, 3, 0.0, 34),            # ceil(100/3) = 34
    (10, 4, 0.5, 4),              # ceil(2.5) = 3, 1.5 * 3 = 4.5
    (1048576, 16, 0.03, 67502),   # 1.03 * 65536 = 67502.08
    (7, 7, 0.0, 1),
])
def test_lmax_closed_form(W, k, eps, want):
    assert O.lmax(W, k, eps) == want


# ------------------------------------------------------------------------------------- LP
def _lp_cases():
    with open(os.path.join(GOLD, "lp_hand.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _lp_cases(), ids=lambda c: c["name"])
def test_lp_hand_traced(case):
    g = _graph(case)
    assert gg.validate(gg.Graph(g.n, g.off, g.adj, None, None if g.ew is None else g.ew.astype(np.int32))) == 0
    labels = np.array(case["labels_in"], dtype=np.int32)
    nl = len(case["lw_out"])
    lw = np.bincount(labels, weights=O.vertex_weights(g), minlength=nl).astype(np.int64)
    for r, bits in case["bits"].items():
        rr = int(r[1:])
        assert [O.hash3(case["seed"], rr, v) >> 63 for v in range(g.n)] == bits
    q = None if case["q"] is None else np.array(case["q"], dtype=np.int32)
    lab, lw2, st = O.lp(g, labels, lw, case["U"], case["rounds"], case["seed"], q)
    assert lab.tolist() == case["labels_out"]
    assert lw2.tolist() == case["lw_out"]
    for key, val in case["stats"].items():
        assert getattr(st, key) == val, key


def _small_graphs():
    gs = [gg.grid(9, 7), gg.rgg(600, 8.0, 3), gg.rmat(9, 8, seed=2), gg.rmat(9, 8, seed=5, weighted=True)]
    g = gg.rgg(500, 10.0, 9)
    rng = np.random.default_rng(4)
    g.vw = rng.integers(1, 4, g.n).astype(np.int64)
    gs.append(g)
    return gs


@pytest.mark.parametrize("gi", range(5))
def test_lp_cluster_invariants(gi):
    g = _small_graphs()[gi]
    c = O.vertex_weights(g)
    U = int(max(c.max(), 6))
    lab, lw, st = O.lp_cluster(g, U, 10, 12345)
    assert lab.min() >= 0 and lab.max() < g.n
    assert np.array_equal(lw, np.bincount(lab, weights=c, minlength=g.n).astype(np.int64))
    assert lw.max() <= U
    assert st.moves > 0 and st.rounds <= 10


@pytest.mark.parametrize("gi", range(5))
def test_lp_first_subround_moves_are_best_eligible(gi):
    """Brute force over the first sub-round: every vertex that moved took a label of maximal
    connection among the eligible labels, with strictly positive gain (Section III-A)."""
    g = _small_graphs()[gi]
    c = O.vertex_weights(g)
    U = int(max(c.max(), 5))
    seed = 99
    lab, _, _ = O.lp_cluster(g, U, 1, seed)
    sub0 = [v for v in range(g.n) if O.hash3(seed, 0, v) >> 63 == 0]
    for v in sub0:
        if lab[v] == v:
            continue
        conn = {}
        for e in range(g.off[v], g.off[v + 1]):
            u = int(g.adj[e])
            conn[u] = conn.get(u, 0) + (1 if g.ew is None else int(g.ew[e]))
        own = conn.get(v, 0)
        best = max(w for L, w in conn.items() if L != v and c[L] + c[v] <= U)
        L = int(lab[v])
        # sub-round 1 vertices never move into a sub-round 0 vertex's label before it is read,
        # so a sub-round 0 mover's final label is its sub-round 0 target.
        assert conn[L] == best and best > own


# ------------------------------------------------------------------------------------- contraction
def _brute_quotient(g, labels):
    used = sorted(set(int(x) for x in labels))
    rank = {L: i for i, L in enumerate(used)}
    W = {}
    cw = [0] * len(used)
    for v in range(g.n):
        cw[rank[int(labels[v])]] += 1 if g.vw is None else int(g.vw[v])
        for e in range(g.off[v], g.off[v + 1]):
            a, b = rank[int(labels[v])], rank[int(labels[g.adj[e]])]
            if a != b:
                W[(a, b)] = W.get((a, b), 0) + (1 if g.ew is None else int(g.ew[e]))
    return len(used), cw, W


@pytest.mark.parametrize("gi", range(5))
def test_contract_matches_bruteforce(gi):
    g = _small_graphs()[gi]
    lab, _, _ = O.lp_cluster(g, 8, 10, 7)
    cg, f2c = O.contract(g, lab)
    n2, cw, W = _brute_quotient(g, lab)
    assert cg.n == n2
    assert cg.vw.tolist() == cw
    got = {}
    for a in range(cg.n):
        row = cg.adj[cg.off[a]:cg.off[a + 1]].tolist()
        assert row == sorted(row) and a not in row
        for e in range(cg.off[a], cg.off[a + 1]):
            got[(a, int(cg.adj[e]))] = int(cg.ew[e])
    assert got == W
    # new id = rank of the label among the used labels (prefix sum over a used-flag array)
    used = np.unique(lab)
    assert np.array_equal(f2c, np.searchsorted(used, lab).astype(np.int32))


@pytest.mark.parametrize("gi", range(5))
def test_contract_totals_and_projection(gi):
    g = _small_graphs()[gi]
    lab, _, _ = O.lp_cluster(g, 8, 10, 3)
    cg, f2c = O.contract(g, lab)
    c = O.vertex_weights(g)
    ew = np.ones(g.m_dir, dtype=np.int64) if g.ew is None else g.ew.astype(np.int64)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    intra = ew[lab[src] == lab[g.adj]].sum()
    assert cg.vw.sum() == c.sum()
    assert cg.ew.sum() == ew.sum() - intra  # total edge weight drops by the intra-cluster weight
    assert gg.validate(gg.Graph(cg.n, cg.off, cg.adj, None, cg.ew.astype(np.int32))) == 0
    rng = np.random.default_rng(gi)
    for k in (2, 5):
        pc = rng.integers(0, k, cg.n).astype(np.int32)
        pf = pc[f2c]
        cut_c, bw_c = O.cut(cg, pc, k)
        cut_f, bw_f = O.cut(g, pf, k)
        assert cut_c == cut_f and np.array_equal(bw_c, bw_f)   # Section III-A


def test_cut_equals_sum_of_crossing_weights():
    g = gg.rmat(8, 8, seed=3, weighted=True)
    rng = np.random.default_rng(0)
    part = rng.integers(0, 4, g.n).astype(np.int32)
    want = sum(w for a, b, w in _edges(g) if part[a] != part[b])
    got, bw = O.cut(g, part, 4)
    assert got == want
    assert bw.tolist() == np.bincount(part, minlength=4).tolist()


# ------------------------------------------------------------------------------------- IP
def _ip():
    with open(os.path.join(GOLD, "ip_hand.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _ip()["bisect"], ids=lambda c: c["name"])
def test_bisect_hand_traced(case):
    g = _graph(case)
    assert O.bisect(g, case["k"], case["s_try"]).tolist() == case["part"]


def test_bisect_unreachable_vertices_come_last():
    # two components: triangle {0,1,2} and edge {3,4}; k=2 puts weight >= 2.5 in side 0.
    off = np.array([0, 2, 4, 6, 7, 8])
    adj = np.array([1, 2, 0, 2, 0, 1, 4, 3], dtype=np.int32)
    g = gg.Graph(5, off, adj)
    for s in range(20):
        start = min(range(5), key=lambda v: (O.hash3(s, 0, v), v))
        part = O.bisect(g, 2, s)
        comp = {0, 1, 2} if start < 3 else {3, 4}
        side0 = {v for v in range(5) if part[v] == 0}
        if comp == {0, 1, 2}:
            assert side0 == {0, 1, 2}
        else:
            # the start's component (weight 2) then the unreachable vertex of smallest id
            assert side0 == {3, 4, 0}


@pytest.mark.parametrize("case", _ip()["repair"], ids=lambda c: c["name"])
def test_repair_hand_traced(case):
    g = _graph(case)
    part, rounds = O.repair(g, np.array(case["part_in"]), case["k"], case["lmax"])
    assert part.tolist() == case["part_out"]
    assert rounds == case["rounds"]


# ------------------------------------------------------------------------------------- partition
def _tiny_graphs():
    out = [gg.grid(3, 4), gg.grid(4, 4), gg.rgg(14, 4.0, 2), gg.rmat(4, 3, seed=9)]
    # weighted cycle of 10
    n = 10
    rows = [sorted([(v - 1) % n, (v + 1) % n]) for v in range(n)]
    off = np.cumsum([0] + [2] * n)
    adj = np.array(sum(rows, []), dtype=np.int32)
    ew = np.array([1 + ((min(v, u) * 7 + max(v, u)) % 3) for v in range(n) for u in rows[v]], dtype=np.int64)
    out.append(gg.Graph(n, off, adj, None, ew))
    return out


@pytest.mark.parametrize("gi", range(5))
def test_partition_tiny_vs_bruteforce_optimum(gi):
    g = _tiny_graphs()[gi]
    k, eps = 2, 0.03
    part, res = O.partition(g, k, eps, seed=1)
    c = O.vertex_weights(g)
    L = O.lmax(int(c.sum()), k, eps)
    edges = _edges(g)
    best = None
    for mask in range(1 << (g.n - 1)):  # vertex n-1 fixed in block 0 (symmetry)
        side = [(mask >> v) & 1 for v in range(g.n)]
        w1 = sum(int(c[v]) for v in range(g.n) if side[v])
        if w1 > L or c.sum() - w1 > L:
            continue
        cutv = sum(w for a, b, w in edges if side[a] != side[b])
        best = cutv if best is None else min(best, cutv)
    cut_o, bw = O.cut(g, part, k)
    assert res.cut == cut_o and res.max_block_weight == bw.max()
    assert best is not None and res.cut >= best
    assert res.imbalanced == 0 and bw.max() <= L
    print(f"{g.name or gi}: oracle cut {res.cut}, optimum {best}, ratio {res.cut / max(best, 1):.2f}")


@pytest.mark.parametrize("gname", ["grid", "rgg", "rmat", "rmatw"])
def test_partition_invariants(gname):
    g = {"grid": lambda: gg.grid(40, 40), "rgg": lambda: gg.rgg(4000, 10.0, 1),
         "rmat": lambda: gg.rmat(12, 8, seed=1), "rmatw": lambda: gg.rmat(11, 8, seed=2, weighted=True)}[gname]()
    k = 4
    params = O.default_params()
    params.coarse_min = 200
    part, res = O.partition(g, k, 0.03, seed=3, params=params)
    assert part.min() >= 0 and part.max() < k
    cut_o, bw = O.cut(g, part, k)
    assert res.cut == cut_o == sum(w for a, b, w in _edges(g) if part[a] != part[b])
    assert res.max_block_weight == bw.max()
    assert res.lmax == O.lmax(int(O.vertex_weights(g).sum()), k, 0.03)
    assert res.imbalanced == int(bw.max() > res.lmax)
    assert res.levels >= 1
    for l in range(res.levels):
        assert res.level_n[l + 1] <= res.level_n[l]


def _waterfill(bw0, count):
    """Closed form of 'each unit-weight vertex to the lightest block, ties to the smaller id':
    at water level x every block with weight <= x receives one vertex per level, in id order."""
    bw0 = list(bw0)
    k = len(bw0)

    def served_before(x):  # vertices handed out before the level reaches x
        return sum(max(0, x - b) for b in bw0)

    out = []
    for j in range(count):
        lo, hi = min(bw0), min(bw0) + count + 1
        while hi - lo > 1:  # largest x with served_before(x) <= j
            mid = (lo + hi) // 2
            if served_before(mid) <= j:
                lo = mid
            else:
                hi = mid
        x = lo
        ids = [b for b in range(k) if bw0[b] <= x]
        out.append(ids[j - served_before(x)])
    return out


def test_partition_isolated_vertices_water_filling():
    base = gg.rgg(300, 6.0, 4)
    iso = np.flatnonzero(np.diff(base.off) == 0)
    # add 40 isolated vertices at the end
    n = base.n + 40
    off = np.concatenate([base.off, np.full(40, base.off[-1])])
    g = gg.Graph(n, off, base.adj)
    k = 3
    part, res = O.partition(g, k, 0.03, seed=2)
    iso = np.flatnonzero(np.diff(g.off) == 0)
    assert res.n_isolated == len(iso)
    keep = np.ones(n, bool)
    keep[iso] = False
    bw0 = np.bincount(part[keep], minlength=k)
    assert part[iso].tolist() == _waterfill(bw0, len(iso))


# ------------------------------------------------------------------------------------- MLP
def _weights(seed=0):
    rng = np.random.default_rng(seed)
    return (rng.normal(0, 0.5, (32, 8)), rng.normal(0, 0.1, 32), rng.normal(0, 0.5, 32), 0.1)


def test_mlp_forward_closed_form():
    # W1 = 0: h = relu(b1) for every row, so s = sigmoid(b2 + sum_j w2_j relu(b1_j)).
    x = np.random.default_rng(1).normal(size=(5, 8))
    _, b1, w2, b2 = _weights(2)
    s = O.mlp_forward(x, np.zeros((32, 8)), b1, w2, b2)
    z = b2 + float(np.dot(w2, np.maximum(b1, 0)))
    assert np.allclose(s, 1 / (1 + math.exp(-z)), rtol=0, atol=1e-15)
    # one hidden unit active: s = sigmoid(w2_0 * (x . W1_0 + b1_0) + b2)
    w1 = np.zeros((32, 8))
    w1[0] = np.arange(1, 9) / 10
    b1z = np.zeros(32)
    w2z = np.zeros(32)
    w2z[0] = 2.0
    xx = np.array([[1.0] * 8, [-1.0] * 8])
    s = O.mlp_forward(xx, w1, b1z, w2z, -1.0)
    assert abs(s[0] - 1 / (1 + math.exp(-(2 * 3.6 - 1)))) < 1e-15
    assert abs(s[1] - 1 / (1 + math.exp(1))) < 1e-15


def test_mlp_gradients_central_differences():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(40, 8))
    y = (rng.random(40) < 0.5).astype(np.float64)
    w1, b1, w2, b2 = _weights(4)
    loss, gw1, gb1, gw2, gb2 = O.mlp_loss_grad(x, y, w1, b1, w2, b2)
    h = 1e-6

    def f(w1_, b1_, w2_, b2_):
        s = O.mlp_forward(x, w1_, b1_, w2_, b2_)
        return float(np.mean(-(y * np.log(s) + (1 - y) * np.log(1 - s))))

    assert abs(loss - f(w1, b1, w2, b2)) < 1e-12
    for idx in [(0, 0), (5, 3), (31, 7), (17, 1)]:
        a, b = w1.copy(), w1.copy()
        a[idx] += h
        b[idx] -= h
        assert abs((f(a, b1, w2, b2) - f(b, b1, w2, b2)) / (2 * h) - gw1[idx]) < 1e-7
    for j in [0, 9, 31]:
        a, b = b1.copy(), b1.copy()
        a[j] += h
        b[j] -= h
        assert abs((f(w1, a, w2, b2) - f(w1, b, w2, b2)) / (2 * h) - gb1[j]) < 1e-7
        a, b = w2.copy(), w2.copy()
        a[j] += h
        b[j] -= h
        assert abs((f(w1, b1, a, b2) - f(w1, b1, b, b2)) / (2 * h) - gw2[j]) < 1e-7
    assert abs((f(w1, b1, w2, b2 + h) - f(w1, b1, w2, b2 - h)) / (2 * h) - gb2) < 1e-7


def test_edge_features_hand_values():
    # triangle 0-1-2 plus pendant 3 attached to 2; edge weights 0-1:1, 0-2:2, 1-2:3, 2-3:4
    off = np.array([0, 2, 4, 7, 8])
    adj = np.array([1, 2, 0, 2, 0, 1, 3, 2], dtype=np.int32)
    ew = np.array([1, 2, 1, 3, 2, 3, 4, 4], dtype=np.int64)
    vw = np.array([1, 2, 3, 4], dtype=np.int64)
    g = gg.Graph(4, off, adj, vw, ew)
    f = O.edge_features(g, level=3)
    # entry 1 is (0,2): d = 2 and 3, c = 1 and 3, w = 2, shared neighbours {1}, wdeg(0)=3, wdeg(2)=9
    want = [math.log2(3), math.log2(4), math.log2(3), math.log2(2), math.log2(4), 1 / 64, 2 / 9, 3 / 16]
    assert np.allclose(f[1], want, atol=1e-15)
    # symmetric: entry 4 is (2,0)
    assert np.array_equal(f[1], f[4])
    # entry 6 is (2,3): d = 3 and 1, no shared neighbours, w=4, wdeg(3)=4
    assert np.allclose(f[6], [1, 2, math.log2(5), math.log2(4), math.log2(5), 0, 4 / 9, 3 / 16], atol=1e-15)
