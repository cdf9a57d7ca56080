"""Pins of the oracle's sequential in-place LP order (``oracle.lp_async``, Section III-A; the order of
Section IV-A's asynchronous form), the comparator for the library's deterministic Jacobi rounds.

* A path worked by hand: the two degree-1 ends come first in the order and join their neighbours'
  clusters at once; the middle vertices then see one neighbour in each cluster (a tie their own label
  wins), and the second iteration moves nothing.
* The size bound: with U equal to the largest vertex weight nothing can move.
* Invariants on random graphs: label weights equal the vertex-weight sums, no cluster exceeds U, every
  label is a vertex id.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O


def test_path_by_hand():
    off = np.array([0, 1, 3, 5, 6], dtype=np.int64)
    adj = np.array([1, 0, 2, 1, 3, 2], dtype=np.int32)
    g = gg.Graph(4, off, adj)
    lab, lw, st = O.lp_cluster_async(g, 10, 10, 1)
    # order (degree, id): 0, 3, 1, 2. Vertex 0 joins 1, vertex 3 joins 2; 1 and 2 each see one
    # neighbour in their own cluster and one in the other (tie: they stay).
    assert list(lab) == [1, 1, 2, 2]
    assert list(lw) == [0, 2, 2, 0]
    assert (st.rounds, st.moves, st.visits, st.edges, st.movers) == (2, 2, 6, 10, 2)


def test_bound_blocks_every_move():
    g = gg.grid(12, 9)
    lab, lw, st = O.lp_cluster_async(g, 1, 10, 3)
    assert np.array_equal(lab, np.arange(g.n)) and st.moves == 0 and st.rounds == 1


@pytest.mark.parametrize("make,U", [(lambda: gg.rgg(5000, 10.0, 2), 30), (lambda: gg.rmat(11, 8, seed=4), 50),
                                    (lambda: gg.grid(40, 40), 7)])
def test_invariants(make, U):
    g = make()
    lab, lw, st = O.lp_cluster_async(g, U, 10, 9)
    c = O.vertex_weights(g)
    assert np.array_equal(np.bincount(lab, weights=c, minlength=g.n).astype(np.int64), lw)
    assert lw.max() <= U and lab.min() >= 0 and lab.max() < g.n
    assert st.moves > 0
