"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded C++ restatement of the partitioner's hot path (size-constrained
label propagation, contraction, initial partitioning, projection and LP refinement of
"High-Quality Shared-Memory Graph Partitioning", Sections III and IV), plus the FP64 edge scorer.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it. It
shares no code with the GPU library; the GPU path never calls it.

Every function takes ``graphgen.Graph`` inputs (host numpy CSR) and returns numpy arrays.
Parity status of each function (what pins it) is listed in ``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

from graphgen import Graph

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRCS = ["lp.cpp", "contract.cpp", "partition.cpp", "mlp.cpp", "match.cpp", "mls.cpp", "lp_async.cpp"]
_lib = None
_lock = threading.Lock()

I64, U64, I32, DBL, VP = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class OrGraph(ctypes.Structure):
    _fields_ = [("n", I64), ("m_dir", I64), ("off", VP), ("adj", VP), ("vw", VP), ("ew", VP)]


class OrLpStats(ctypes.Structure):
    _fields_ = [("rounds", I64), ("moves", I64), ("visits", I64), ("edges", I64), ("movers", I64)]


class OrParams(ctypes.Structure):
    _fields_ = [("cluster_div", I64), ("rounds_coarsen", I64), ("rounds_refine", I64),
                ("coarse_min", I64), ("coarse_per_k", I64), ("stall_pct", I64),
                ("max_levels", I64), ("ip_tries", I64), ("repair_rounds", I64), ("coarsen_mode", I64),
                ("mls", I64), ("lp_async", I64)]


class OrMlsParams(ctypes.Structure):
    _fields_ = [("global_iters", I64), ("alpha_pct", I64), ("max_local", I64), ("max_moves", I64),
                ("fruitless", I64), ("queue_cap", I64), ("max_degree", I64)]


class OrMlsStats(ctypes.Structure):
    _fields_ = [("gain", I64), ("moves", I64), ("searches", I64), ("local_iters", I64)]


class OrMatchStats(ctypes.Structure):
    _fields_ = [("rounds", I64), ("pairs", I64)]


class OrResult(ctypes.Structure):
    _fields_ = [("cut", I64), ("max_block_weight", I64), ("lmax", I64), ("imbalanced", I64),
                ("levels", I64), ("best_try", I64), ("n_isolated", I64),
                ("level_n", I64 * 65), ("level_m", I64 * 65),
                ("try_cut", I64 * 16), ("try_imbalanced", I64 * 16), ("lp_edges", I64)]


def build(force: bool = False) -> str:
    """Compile the oracle sources into liboracle.so with g++ (-O2, single-threaded)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", *srcs, "-o", _LIB + ".tmp"],
                   check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.or_mix64.restype = U64
            lib.or_mix64.argtypes = [U64]
            lib.or_hash3.restype = U64
            lib.or_hash3.argtypes = [U64, U64, U64]
            lib.or_lmax.restype = I64
            lib.or_lmax.argtypes = [I64, I64, DBL]
            lib.or_lp.restype = I32
            lib.or_lp.argtypes = [ctypes.POINTER(OrGraph), VP, VP, VP, I64, I64, I64, U64,
                                  ctypes.POINTER(OrLpStats)]
            lib.or_contract.restype = I32
            lib.or_contract.argtypes = [ctypes.POINTER(OrGraph), VP, I64, ctypes.POINTER(I64),
                                        ctypes.POINTER(I64), VP, VP, VP, VP, VP]
            lib.or_lp_async.restype = I32
            lib.or_lp_async.argtypes = [ctypes.POINTER(OrGraph), VP, VP, I64, I64, I64, U64, ctypes.POINTER(OrLpStats)]
            lib.or_match.restype = I32
            lib.or_match.argtypes = [ctypes.POINTER(OrGraph), I64, I64, U64, VP, ctypes.POINTER(OrMatchStats)]
            lib.or_mls_default_params.restype = None
            lib.or_mls_default_params.argtypes = [ctypes.POINTER(OrMlsParams)]
            lib.or_mls.restype = I64
            lib.or_mls.argtypes = [ctypes.POINTER(OrGraph), I64, I64, U64, ctypes.POINTER(OrMlsParams), VP,
                                   ctypes.POINTER(OrMlsStats)]
            lib.or_bisect.restype = I32
            lib.or_bisect.argtypes = [ctypes.POINTER(OrGraph), I64, U64, VP]
            lib.or_repair.restype = I64
            lib.or_repair.argtypes = [ctypes.POINTER(OrGraph), I64, I64, I64, VP]
            lib.or_cut.restype = I64
            lib.or_cut.argtypes = [ctypes.POINTER(OrGraph), VP, I64, VP]
            lib.or_default_params.restype = None
            lib.or_default_params.argtypes = [ctypes.POINTER(OrParams)]
            lib.or_partition.restype = I32
            lib.or_partition.argtypes = [ctypes.POINTER(OrGraph), I64, DBL, U64,
                                         ctypes.POINTER(OrParams), VP, I64, VP,
                                         ctypes.POINTER(OrResult)]
            lib.or_edge_features.restype = None
            lib.or_edge_features.argtypes = [ctypes.POINTER(OrGraph), I64, VP]
            lib.or_mlp_forward.restype = None
            lib.or_mlp_forward.argtypes = [I64, VP, VP, VP, VP, DBL, VP]
            lib.or_mlp_loss_grad.restype = DBL
            lib.or_mlp_loss_grad.argtypes = [I64, VP, VP, VP, VP, VP, DBL, VP, VP, VP, VP]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


class _View:
    """Holds int64 copies of a Graph's arrays alive while the oracle reads them."""

    def __init__(self, g: Graph):
        self.off = np.ascontiguousarray(g.off, dtype=np.int64)
        self.adj = np.ascontiguousarray(g.adj, dtype=np.int32)
        self.vw = None if g.vw is None else np.ascontiguousarray(g.vw, dtype=np.int64)
        self.ew = None if g.ew is None else np.ascontiguousarray(g.ew, dtype=np.int64)
        self.s = OrGraph(g.n, int(self.adj.shape[0]), _p(self.off), _p(self.adj), _p(self.vw), _p(self.ew))

    def ref(self):
        return ctypes.byref(self.s)


def mix64(z: int) -> int:
    return int(_load().or_mix64(z))


def hash3(a: int, b: int, c: int) -> int:
    return int(_load().or_hash3(a, b, c))


def lmax(total_weight: int, k: int, eps: float) -> int:
    return int(_load().or_lmax(total_weight, k, eps))


def vertex_weights(g: Graph) -> np.ndarray:
    return np.ones(g.n, dtype=np.int64) if g.vw is None else np.asarray(g.vw, dtype=np.int64)


@dataclass
class LpStats:
    rounds: int
    moves: int
    visits: int
    edges: int
    movers: int


def lp(g: Graph, labels, lw, U: int, rounds: int, seed: int, q=None):
    """One LP run from (labels, label weights); returns (labels, lw, LpStats)."""
    v = _View(g)
    labels = np.array(labels, dtype=np.int32, copy=True)
    lw = np.array(lw, dtype=np.int64, copy=True)
    qa = None if q is None else np.ascontiguousarray(q, dtype=np.int32)
    st = OrLpStats()
    rc = _load().or_lp(v.ref(), _p(qa), _p(labels), _p(lw), int(lw.shape[0]), U, rounds, seed,
                       ctypes.byref(st))
    assert rc == 0
    return labels, lw, LpStats(st.rounds, st.moves, st.visits, st.edges, st.movers)


def lp_cluster(g: Graph, U: int, rounds: int, seed: int, q=None):
    """Size-constrained LP clustering from singletons (C[v] = v)."""
    return lp(g, np.arange(g.n, dtype=np.int32), vertex_weights(g), U, rounds, seed, q)


def lp_async(g: Graph, labels, lw, U: int, rounds: int, seed: int):
    """The paper's sequential in-place LP order ((degree, id) order, moves applied at once)."""
    v = _View(g)
    labels = np.array(labels, dtype=np.int32, copy=True)
    lw = np.array(lw, dtype=np.int64, copy=True)
    st = OrLpStats()
    rc = _load().or_lp_async(v.ref(), _p(labels), _p(lw), int(lw.shape[0]), U, rounds, seed, ctypes.byref(st))
    assert rc == 0
    return labels, lw, LpStats(st.rounds, st.moves, st.visits, st.edges, st.movers)


def lp_cluster_async(g: Graph, U: int, rounds: int, seed: int):
    return lp_async(g, np.arange(g.n, dtype=np.int32), vertex_weights(g), U, rounds, seed)


def block_weights(g: Graph, part, k: int) -> np.ndarray:
    return np.bincount(np.asarray(part, dtype=np.int64), weights=vertex_weights(g), minlength=k).astype(np.int64)


def lp_refine(g: Graph, part, k: int, lmax_: int, rounds: int, seed: int):
    """LP refinement of a k-way partition under U = Lmax."""
    return lp(g, part, block_weights(g, part, k), lmax_, rounds, seed)


def contract(g: Graph, labels, nl: int | None = None):
    """Quotient graph of a clustering; returns (coarse Graph with int64 weights, f2c int32[n])."""
    v = _View(g)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    nl = g.n if nl is None else nl
    off = np.zeros(g.n + 1, dtype=np.int64)
    adj = np.zeros(max(g.m_dir, 1), dtype=np.int32)
    vw = np.zeros(max(g.n, 1), dtype=np.int64)
    ew = np.zeros(max(g.m_dir, 1), dtype=np.int64)
    f2c = np.zeros(g.n, dtype=np.int32)
    nn, mm = I64(0), I64(0)
    rc = _load().or_contract(v.ref(), _p(labels), nl, ctypes.byref(nn), ctypes.byref(mm), _p(off),
                             _p(adj), _p(vw), _p(ew), _p(f2c))
    assert rc == 0
    n2, m2 = nn.value, mm.value
    return Graph(n2, off[: n2 + 1].copy(), adj[:m2].copy(), vw[:n2].copy(), ew[:m2].copy(), "coarse"), f2c


def match(g: Graph, U: int, rounds: int, seed: int):
    """Matching-based clustering (handshake matching, clusters of one or two vertices); returns
    (labels int32[n], {"rounds", "pairs"})."""
    v = _View(g)
    labels = np.zeros(g.n, dtype=np.int32)
    st = OrMatchStats()
    rc = _load().or_match(v.ref(), U, rounds, seed, _p(labels), ctypes.byref(st))
    assert rc == 0
    return labels, {"rounds": st.rounds, "pairs": st.pairs}


def mls_default_params() -> OrMlsParams:
    p = OrMlsParams()
    _load().or_mls_default_params(ctypes.byref(p))
    return p


def mls(g: Graph, part, k: int, lmax_: int, seed: int, params: OrMlsParams | None = None):
    """Multi-try k-way local search on a copy of `part`; returns (part, stats dict)."""
    v = _View(g)
    part = np.array(part, dtype=np.int32, copy=True)
    st = OrMlsStats()
    _load().or_mls(v.ref(), k, lmax_, seed, ctypes.byref(params) if params else None, _p(part), ctypes.byref(st))
    return part, {"gain": st.gain, "moves": st.moves, "searches": st.searches, "local_iters": st.local_iters}


def bisect(g: Graph, k: int, s_try: int) -> np.ndarray:
    v = _View(g)
    part = np.zeros(g.n, dtype=np.int32)
    _load().or_bisect(v.ref(), k, s_try, _p(part))
    return part


def repair(g: Graph, part, k: int, lmax_: int, max_rounds: int = 16):
    v = _View(g)
    part = np.array(part, dtype=np.int32, copy=True)
    rounds = _load().or_repair(v.ref(), k, lmax_, max_rounds, _p(part))
    return part, int(rounds)


def cut(g: Graph, part, k: int):
    """Returns (cut, block weights)."""
    v = _View(g)
    part = np.ascontiguousarray(part, dtype=np.int32)
    bw = np.zeros(k, dtype=np.int64)
    c = _load().or_cut(v.ref(), _p(part), k, _p(bw))
    return int(c), bw


def default_params() -> OrParams:
    p = OrParams()
    _load().or_default_params(ctypes.byref(p))
    return p


def partition(g: Graph, k: int, eps: float, seed: int, params: OrParams | None = None, q_levels=None):
    """Full multilevel partition; returns (part int32[n], OrResult)."""
    v = _View(g)
    part = np.zeros(g.n, dtype=np.int32)
    res = OrResult()
    qarr, keep = None, []
    nq = 0
    if q_levels is not None:
        keep = [np.ascontiguousarray(q, dtype=np.int32) for q in q_levels]
        qarr = (VP * max(len(keep), 1))(*[q.ctypes.data for q in keep])
        nq = len(keep)
    rc = _load().or_partition(v.ref(), k, eps, seed, ctypes.byref(params) if params else None,
                              ctypes.cast(qarr, VP) if qarr is not None else None, nq, _p(part),
                              ctypes.byref(res))
    if rc != 0:
        raise ValueError(f"oracle partition rejected its input (code {rc})")
    return part, res


def edge_features(g: Graph, level: int) -> np.ndarray:
    v = _View(g)
    feat = np.zeros((g.m_dir, 8), dtype=np.float64)
    _load().or_edge_features(v.ref(), level, _p(feat))
    return feat


def mlp_forward(x, w1, b1, w2, b2) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    w1, b1, w2 = (np.ascontiguousarray(a, dtype=np.float64) for a in (w1, b1, w2))
    s = np.zeros(x.shape[0], dtype=np.float64)
    _load().or_mlp_forward(x.shape[0], _p(x), _p(w1), _p(b1), _p(w2), float(b2), _p(s))
    return s


def mlp_loss_grad(x, y, w1, b1, w2, b2):
    """Mean BCE and gradients (gw1[32,8], gb1[32], gw2[32], gb2)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    w1, b1, w2 = (np.ascontiguousarray(a, dtype=np.float64) for a in (w1, b1, w2))
    gw1 = np.zeros((32, 8))
    gb1 = np.zeros(32)
    gw2 = np.zeros(32)
    gb2 = ctypes.c_double(0.0)
    loss = _load().or_mlp_loss_grad(x.shape[0], _p(x), _p(y), _p(w1), _p(b1), _p(w2), float(b2),
                                    _p(gw1), _p(gb1), _p(gw2), ctypes.byref(gb2))
    return float(loss), gw1, gb1, gw2, float(gb2.value)
