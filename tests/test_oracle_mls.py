"""Pins of the oracle's multi-try k-way local search (``oracle.mls``, Sections III-C and IV-C).

* Two cases worked by hand in which no hash decides the outcome:
  - a path where one vertex sits alone in the other block: every search finds the same single move
    (gain 2), the first sequence applies it, the others stop at the moved vertex;
  - two heavily joined vertices that only pay off together (each single move has gain -3, the pair
    has gain +4: the search must accept the negative first move and keep the best prefix), with the
    balance bound blocking every other move.
* Invariants on random partitions: the reported gain equals the cut before minus the cut after, the
  cut never grows, no block goes above Lmax, vertices above the degree bound never move, and with
  zero global iterations nothing changes.
* In the partition driver (mls != 0) the result equals the step-by-step restatement that calls the
  pinned primitives (tests/test_oracle_driver.py).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O


def _from_edges(n, edges):
    e = sorted([(u, v, w) for u, v, w in edges] + [(v, u, w) for u, v, w in edges])
    off = np.zeros(n + 1, dtype=np.int64)
    for u, _, _ in e:
        off[u + 1] += 1
    return gg.Graph(n, np.cumsum(off), np.array([v for _, v, _ in e], dtype=np.int32), None,
                    np.array([w for _, _, w in e], dtype=np.int64))


def test_single_improving_move_by_hand():
    # path 0-1-2-3-4-5, vertex 2 alone in block 1: moving it to block 0 gains 2 (both its edges)
    g = _from_edges(6, [(i, i + 1, 1) for i in range(5)])
    part = np.array([0, 0, 1, 0, 0, 0], dtype=np.int32)
    lmax = O.lmax(6, 2, 1.0)  # floor(2 * 3) = 6: block 0 may take all six
    out, st = O.mls(g, part, 2, lmax, 7)
    assert list(out) == [0] * 6
    # first global iteration: searches from the boundary vertices 1, 2, 3, then one search from the
    # moved vertex 2 that finds nothing; the later global iterations have no boundary vertex
    assert st == {"gain": 2, "moves": 1, "searches": 4, "local_iters": 2}


def test_negative_first_move_pays_off_by_hand():
    # A = {0,1,2,3,4}, B = {5,6,7}. 0 and 1 share an edge of weight 5; each has weight 3 to B and 1 to
    # an A vertex anchored by weight 10. Moving 0 or 1 alone gains 3 - 6 = -3; after one moved, the
    # other gains 8 - 1 = 7: the pair gains 4. Lmax = 5 keeps B from growing beyond the pair and A
    # (weight 5) from taking any B vertex.
    edges = [(0, 1, 5), (0, 2, 1), (1, 3, 1), (0, 5, 3), (1, 6, 3), (2, 4, 10), (3, 4, 10), (5, 7, 10), (6, 7, 10)]
    g = _from_edges(8, edges)
    part = np.array([0, 0, 0, 0, 0, 1, 1, 1], dtype=np.int32)
    lmax = O.lmax(8, 2, 0.25)
    assert lmax == 5
    before, _ = O.cut(g, part, 2)
    out, st = O.mls(g, part, 2, lmax, 3)
    after, bw = O.cut(g, out, 2)
    assert (before, after) == (6, 2)
    assert list(out) == [1, 1, 0, 0, 0, 1, 1, 1]
    assert st["gain"] == 4 and st["moves"] == 2
    assert bw.max() <= lmax


def _random_case(seed, n=3000, k=8):
    g = gg.rgg(n, 9.0, seed)
    rng = np.random.default_rng(seed)
    if seed % 2:
        g.vw = rng.integers(1, 4, g.n).astype(np.int64)
        src = np.repeat(np.arange(g.n), np.diff(g.off))
        lo, hi = np.minimum(src, g.adj), np.maximum(src, g.adj)
        g.ew = (1 + (lo * 31 + hi * 17) % 5).astype(np.int64)
    c = O.vertex_weights(g)
    lmax = O.lmax(int(c.sum()), k, 0.03)
    # a balanced start: an LP-refined partition of the graph
    part, _ = O.partition(g, k, 0.03, seed)
    return g, part, k, lmax


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_mls_invariants(seed):
    g, part, k, lmax = _random_case(seed)
    before, bw0 = O.cut(g, part, k)
    assert bw0.max() <= lmax
    out, st = O.mls(g, part, k, lmax, 11 + seed)
    after, bw = O.cut(g, out, k)
    assert st["gain"] == before - after >= 0
    assert bw.max() <= lmax and bw.sum() == bw0.sum()
    assert np.count_nonzero(out != part) <= st["moves"]
    # nothing happens without global iterations
    p = O.mls_default_params()
    p.global_iters = 0
    same, st0 = O.mls(g, part, k, lmax, 1, p)
    assert np.array_equal(same, part) and st0["gain"] == 0


def test_mls_degree_bound():
    g = gg.rmat(11, 8, seed=5)
    k = 4
    lmax = O.lmax(g.n, k, 0.03)
    part, _ = O.partition(g, k, 0.03, 2)
    p = O.mls_default_params()
    p.max_degree = 20
    out, st = O.mls(g, part, k, lmax, 9, p)
    deg = np.diff(g.off)
    assert np.array_equal(out[deg > 20], part[deg > 20])
    assert st["gain"] == O.cut(g, part, k)[0] - O.cut(g, out, k)[0]
