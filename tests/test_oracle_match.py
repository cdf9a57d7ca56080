"""Pins of the oracle's matching-based clustering (``oracle.match``).

* Two cases worked by hand (no hash decides them): a path whose middle edge is heaviest, and a star
  whose centre must pick the leaf of best rating omega^2 / (c(u) c(v)), with one leaf excluded by U.
* Brute force: with a strict order on edges that is the same seen from both endpoints, handshake
  matching run to convergence gives exactly the greedy matching that scans all edges once in
  decreasing order (a classical fact about locally dominant edges, Preis 1999). The greedy matching
  is computed here from an explicit sorted edge list with exact rational ratings.
* Invariants: clusters of one or two adjacent vertices, the bound U holds, and a run that stopped
  because a round matched nothing leaves no unmatched adjacent pair that fits U (maximality).
"""
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle as O


def _from_edges(n, edges, vw=None):
    e = sorted([(u, v, w) for u, v, w in edges] + [(v, u, w) for u, v, w in edges])
    off = np.zeros(n + 1, dtype=np.int64)
    for u, _, _ in e:
        off[u + 1] += 1
    off = np.cumsum(off)
    adj = np.array([v for _, v, _ in e], dtype=np.int32)
    ew = np.array([w for _, _, w in e], dtype=np.int64)
    return gg.Graph(n, off, adj, None if vw is None else np.array(vw, dtype=np.int64), ew)


def test_path_heavy_middle_edge_by_hand():
    # 0 -1- 1 -5- 2 -1- 3: vertices 1 and 2 propose to each other (rating 25 against 1); 0 and 3 propose
    # to them and stay alone; the next round has no unmatched neighbour left for 0 or 3
    g = _from_edges(4, [(0, 1, 1), (1, 2, 5), (2, 3, 1)])
    lab, st = O.match(g, 10, 8, 99)
    assert list(lab) == [0, 1, 1, 3]
    assert st == {"rounds": 2, "pairs": 1}


def test_star_rating_and_bound_by_hand():
    # centre 0 (c=1); leaves 1 (c=5, w=3): 9/5; 2 (c=1, w=2): 4; 3 (c=2, w=3): 9/2; 4 (c=9, w=9): 81/9 = 9
    # but 1 + 9 > U = 6, so leaf 4 is not eligible and the centre picks leaf 3
    g = _from_edges(5, [(0, 1, 3), (0, 2, 2), (0, 3, 3), (0, 4, 9)], vw=[1, 5, 1, 2, 9])
    lab, st = O.match(g, 6, 8, 5)
    assert list(lab) == [0, 1, 2, 0, 4]
    assert st["pairs"] == 1
    # with U = 10 leaf 4 (rating 9) wins
    lab, _ = O.match(g, 10, 8, 5)
    assert list(lab) == [0, 1, 2, 3, 0]


def _greedy(g, U, seed):
    vw = O.vertex_weights(g)
    edges = []
    for v in range(g.n):
        for e in range(g.off[v], g.off[v + 1]):
            u = int(g.adj[e])
            if v < u:
                w = 1 if g.ew is None else int(g.ew[e])
                edges.append((Fraction(w * w, int(vw[u] * vw[v])), O.hash3(seed, v, u), v, u))
    edges.sort(key=lambda x: (x[0], x[1]), reverse=True)
    mate = [-1] * g.n
    for _, _, v, u in edges:
        if mate[v] < 0 and mate[u] < 0 and vw[v] + vw[u] <= U:
            mate[v], mate[u] = u, v
    return np.array([min(v, mate[v]) if mate[v] >= 0 else v for v in range(g.n)], dtype=np.int32)


def _weighted_rgg(n, seed):
    g = gg.rgg(n, 7.0, seed)
    rng = np.random.default_rng(seed)
    g.vw = rng.integers(1, 6, g.n).astype(np.int64)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    lo, hi = np.minimum(src, g.adj), np.maximum(src, g.adj)
    g.ew = (1 + (lo * 7919 + hi * 104729) % 9).astype(np.int64)  # symmetric weights in [1, 9]
    return g


@pytest.mark.parametrize("make,U", [(lambda: gg.grid(9, 11), 2), (lambda: gg.rmat(9, 6, seed=4), 2),
                                    (lambda: _weighted_rgg(600, 3), 7), (lambda: _weighted_rgg(900, 8), 5)])
@pytest.mark.parametrize("seed", [1, 77])
def test_converged_handshake_equals_greedy_matching(make, U, seed):
    g = make()
    lab, st = O.match(g, U, 1000, seed)
    assert st["rounds"] < 1000  # ran to convergence
    assert np.array_equal(lab, _greedy(g, U, seed))


@pytest.mark.parametrize("rounds", [1, 2, 3, 50])
def test_matching_invariants(rounds):
    g = _weighted_rgg(1500, 11)
    U = 6
    lab, st = O.match(g, U, rounds, 3)
    vw = O.vertex_weights(g)
    members = {}
    for v, L in enumerate(lab):
        members.setdefault(int(L), []).append(v)
    nbr = [set(g.adj[g.off[v]:g.off[v + 1]].tolist()) for v in range(g.n)]
    pairs = 0
    for L, ms in members.items():
        assert len(ms) <= 2 and L == min(ms)
        if len(ms) == 2:
            a, b = ms
            assert b in nbr[a] and vw[a] + vw[b] <= U
            pairs += 1
    assert pairs == st["pairs"]
    if st["rounds"] < rounds:  # stopped because a round matched nothing: maximal
        single = {ms[0] for ms in members.values() if len(ms) == 1}
        for v in single:
            assert not any(u in single and vw[u] + vw[v] <= U for u in nbr[v])
