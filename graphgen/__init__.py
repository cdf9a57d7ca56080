"""Seeded synthetic input graphs shared by the CPU oracle and the GPU path.

This module generates inputs only; it holds no step of the partitioning method. Graphs are
symmetric CSR (int64 offsets, int32 sorted adjacency, no self-loops), built by ``graphgen.c``.

Families (stand-ins for the paper's benchmark classes of Section VI, Table I, whose files are
not available here):

* ``grid(a, b)``        -- 4-neighbour grid, mesh-like
* ``rgg(n, deg, seed)`` -- random geometric graph in the unit square (the paper's rgg family)
* ``rmat(scale, ...)``  -- R-MAT power-law graph, symmetrised and deduplicated
* ``batch_specs(...)``  -- the uneven mix of grids and rggs used for batched partitioning
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so (OpenMP when the compiler supports it)."""
    src = os.path.join(_HERE, "graphgen.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            vp, i64, u64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            lib.gg_grid.restype = vp
            lib.gg_grid.argtypes = [i64, i64]
            lib.gg_rgg.restype = vp
            lib.gg_rgg.argtypes = [i64, dbl, u64]
            lib.gg_rmat.restype = vp
            lib.gg_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32]
            lib.gg_n.restype = i64
            lib.gg_n.argtypes = [vp]
            lib.gg_m.restype = i64
            lib.gg_m.argtypes = [vp]
            lib.gg_weighted.restype = i32
            lib.gg_weighted.argtypes = [vp]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [vp, vp, vp, vp]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [vp]
            lib.gg_validate.restype = i32
            lib.gg_validate.argtypes = [i64, vp, vp, vp]
            lib.gg_word.restype = u64
            lib.gg_word.argtypes = [u64, u64]
            lib.gg_key3.restype = u64
            lib.gg_key3.argtypes = [u64, u64, u64]
            lib.gg_unif.restype = dbl
            lib.gg_unif.argtypes = [u64, u64]
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Host CSR graph. ``vw``/``ew`` of ``None`` mean unit weights."""

    n: int
    off: np.ndarray  # int64[n+1]
    adj: np.ndarray  # int32[m_dir]
    vw: Optional[np.ndarray] = None  # int32 or int64 [n]
    ew: Optional[np.ndarray] = None  # int32 or int64 [m_dir]
    name: str = ""

    @property
    def m_dir(self) -> int:
        return int(self.adj.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off)


def _take(h, name: str) -> Graph:
    lib = _load()
    n, m = lib.gg_n(h), lib.gg_m(h)
    off = np.empty(n + 1, dtype=np.int64)
    adj = np.empty(max(m, 0), dtype=np.int32)
    ew = np.empty(m, dtype=np.int32) if lib.gg_weighted(h) else None
    lib.gg_copy(h, off.ctypes.data, adj.ctypes.data, ew.ctypes.data if ew is not None else None)
    lib.gg_free(h)
    return Graph(int(n), off, adj, None, ew, name)


def grid(a: int, b: int) -> Graph:
    """a x b 4-neighbour grid; vertex id = row*b + col; unit weights."""
    return _take(_load().gg_grid(a, b), f"grid{a}x{b}")


def rgg(n: int, avg_deg: float = 12.0, seed: int = 1) -> Graph:
    """Random geometric graph: point i at (U(seed,2i), U(seed,2i+1)); edge iff distance < r,
    r = sqrt(avg_deg / (pi n)); ids in generation order; unit weights."""
    return _take(_load().gg_rgg(n, float(avg_deg), seed), f"rgg{n}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, weighted: bool = False) -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor*2^scale samples; symmetrised,
    deduplicated, self-loops removed; integer edge weights in [1,8] when ``weighted``."""
    h = _load().gg_rmat(scale, edge_factor, a, b, c, seed, 1 if weighted else 0)
    return _take(h, f"rmat{scale}{'w' if weighted else ''}")


def validate(g: Graph) -> int:
    """0 when ``g`` is a valid symmetric CSR with equal weights both ways."""
    ew = None
    if g.ew is not None:
        ew = np.ascontiguousarray(g.ew, dtype=np.int32)
    off = np.ascontiguousarray(g.off, dtype=np.int64)
    adj = np.ascontiguousarray(g.adj, dtype=np.int32)
    return int(_load().gg_validate(g.n, off.ctypes.data, adj.ctypes.data,
                                   ew.ctypes.data if ew is not None else None))


def word(seed: int, ctr: int) -> int:
    return int(_load().gg_word(seed, ctr))


def key3(a: int, b: int, c: int) -> int:
    return int(_load().gg_key3(a, b, c))


def unif(seed: int, ctr: int) -> float:
    return float(_load().gg_unif(seed, ctr))


@dataclass
class BatchSpec:
    kind: str  # "grid" or "rgg"
    n: int
    k: int
    seed: int


def batch_specs(count: int = 512, seed: int = 1, n_lo: float = 1e3, n_hi: float = 2e5) -> list:
    """Uneven batch: n_i = round(exp(U[ln n_lo, ln n_hi])), kind by one bit of the graph's key,
    k_i from {2,4,8} by the key mod 3, per-graph seed = key3(seed, i, 0)."""
    out = []
    lo, hi = math.log(n_lo), math.log(n_hi)
    for i in range(count):
        u = unif(seed, i)
        n = int(round(math.exp(lo + u * (hi - lo))))
        key = key3(seed, i, 1)
        kind = "grid" if (key >> 63) & 1 else "rgg"
        k = (2, 4, 8)[key % 3]
        out.append(BatchSpec(kind, n, k, key3(seed, i, 0)))
    return out


def batch_graph(spec: BatchSpec) -> Graph:
    if spec.kind == "grid":
        a = int(math.isqrt(spec.n))
        b = -(-spec.n // a)
        g = grid(a, b)
    else:
        g = rgg(spec.n, 12.0, spec.seed)
    return g
