"""Python binding of the GB300 partitioner C ABI (``include/gpart.h``, ``libgpart.so``).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels. Device
memory and streams come from PyTorch; the library's temporary allocations are routed to PyTorch's
caching allocator through ``gp_set_allocator``. There is no CPU fallback: importing the binding on a
machine without the built library or without a CUDA device raises when a call is made.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpart.so")

I64, U64, I32, DBL, VP, SZ = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                              ctypes.c_void_p, ctypes.c_size_t)

GP_OK, GP_ERR_INVALID_ARG, GP_ERR_BAD_GRAPH, GP_ERR_OOM, GP_ERR_CUDA, GP_ERR_TIMEOUT, GP_ERR_INTERNAL, \
    GP_ERR_UNSUPPORTED = range(8)
MODE_PLAIN, MODE_LEARNED, MODE_BEST_OF = 0, 1, 2
COARSEN_LP, COARSEN_MATCHING = 0, 1


class GpGraph(ctypes.Structure):
    _fields_ = [("n", I64), ("m_dir", I64), ("offsets", VP), ("adj", VP), ("vwgt", VP), ("ewgt", VP),
                ("offsets_64", I32), ("vwgt_64", I32), ("ewgt_64", I32), ("reserved", I32)]


class GpLpStats(ctypes.Structure):
    _fields_ = [("rounds", I64), ("moves", I64), ("visits", I64), ("edges", I64), ("movers", I64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GpMatchStats(ctypes.Structure):
    _fields_ = [("rounds", I64), ("pairs", I64), ("visits", I64), ("edges", I64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GpParams(ctypes.Structure):
    _fields_ = [("cluster_div", I64), ("rounds_coarsen", I64), ("rounds_refine", I64), ("coarse_min", I64),
                ("coarse_per_k", I64), ("stall_pct", I64), ("max_levels", I64), ("ip_tries", I64),
                ("repair_rounds", I64), ("mode", I32), ("deg_warp", I32), ("deg_cta", I32), ("coarsen", I32),
                ("mlp", VP), ("hub_batch_slots", I64), ("verts_per_block", I64), ("mls_global_iters", I64),
                ("lp_async", I64), ("hub_keep_slots", I64)]


class GpMlsParams(ctypes.Structure):
    _fields_ = [("global_iters", I64), ("alpha_pct", I64), ("max_local", I64), ("max_moves", I64),
                ("fruitless", I64), ("queue_cap", I64), ("max_degree", I64)]


class GpMlsStats(ctypes.Structure):
    _fields_ = [("gain", I64), ("moves", I64), ("searches", I64), ("local_iters", I64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GpResult(ctypes.Structure):
    _fields_ = [("cut", I64), ("max_block_weight", I64), ("lmax", I64), ("imbalanced", I64), ("levels", I64),
                ("best_try", I64), ("n_isolated", I64), ("level_n", I64 * 65), ("level_m", I64 * 65),
                ("try_cut", I64 * 16), ("try_imbalanced", I64 * 16), ("lp_edges", I64), ("lp_moves", I64),
                ("plain_cut", I64), ("learned_cut", I64), ("ms_total", DBL), ("ms_coarsen", DBL),
                ("ms_initial", DBL), ("ms_refine", DBL)]


class GpProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", I64), ("ms", DBL), ("items", I64), ("edges", I64),
                ("bytes", I64)]


class GpBatchItem(ctypes.Structure):
    _fields_ = [("g", GpGraph), ("k", I32), ("reserved", I32), ("eps", DBL), ("seed", U64), ("part_out", VP)]


ALLOC_FN = ctypes.CFUNCTYPE(VP, SZ, VP, VP)
FREE_FN = ctypes.CFUNCTYPE(None, VP, SZ, VP, VP)

_lib = None
_lock = threading.Lock()
_keep = []  # ctypes callbacks must outlive the library's use of them
alloc_calls = [0]  # number of allocations the library requested through the installed allocator


class GpError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


def build(force: bool = False) -> str:
    """Compiles libgpart.so in-tree for sm_103a (see buildlib.py)."""
    from . import buildlib
    return buildlib.build(force=force)


def lib():
    """Loads libgpart.so (it must have been built with ``build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first (no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        L.gp_version.restype = ctypes.c_char_p
        L.gp_status_string.restype = ctypes.c_char_p
        L.gp_status_string.argtypes = [ctypes.c_int]
        L.gp_last_error.restype = ctypes.c_char_p
        L.gp_set_allocator.restype = ctypes.c_int
        L.gp_set_allocator.argtypes = [VP, VP, VP]
        L.gp_default_params.restype = None
        L.gp_default_params.argtypes = [ctypes.POINTER(GpParams)]
        L.gp_validate_graph.restype = ctypes.c_int
        L.gp_validate_graph.argtypes = [ctypes.POINTER(GpGraph), VP]
        L.gp_lmax.restype = I64
        L.gp_lmax.argtypes = [I64, I64, DBL]
        L.gp_lp_cluster.restype = ctypes.c_int
        L.gp_lp_cluster.argtypes = [ctypes.POINTER(GpGraph), I64, I32, U64, VP, VP, ctypes.POINTER(GpLpStats), VP]
        L.gp_lp_cluster_noalloc.restype = ctypes.c_int
        L.gp_lp_cluster_noalloc.argtypes = [ctypes.POINTER(GpGraph), I64, I32, U64, VP, VP,
                                            ctypes.POINTER(GpLpStats), VP]
        L.gp_mls_default_params.restype = None
        L.gp_mls_default_params.argtypes = [ctypes.POINTER(GpMlsParams)]
        L.gp_mls.restype = ctypes.c_int
        L.gp_mls.argtypes = [ctypes.POINTER(GpGraph), I32, I64, U64, ctypes.POINTER(GpMlsParams), VP,
                             ctypes.POINTER(GpMlsStats), VP]
        L.gp_lp_cluster_async.restype = ctypes.c_int
        L.gp_lp_cluster_async.argtypes = [ctypes.POINTER(GpGraph), I64, I32, U64, I32, VP, ctypes.POINTER(GpLpStats),
                                          VP]
        L.gp_match.restype = ctypes.c_int
        L.gp_match.argtypes = [ctypes.POINTER(GpGraph), I64, I32, U64, VP, ctypes.POINTER(GpMatchStats), VP]
        L.gp_lp_refine.restype = ctypes.c_int
        L.gp_lp_refine.argtypes = [ctypes.POINTER(GpGraph), I32, I64, I32, U64, VP, VP, ctypes.POINTER(GpLpStats), VP]
        L.gp_contract.restype = ctypes.c_int
        L.gp_contract.argtypes = [ctypes.POINTER(GpGraph), VP, ctypes.POINTER(VP), VP, VP]
        L.gp_coarse_graph.restype = ctypes.POINTER(GpGraph)
        L.gp_coarse_graph.argtypes = [VP]
        L.gp_coarse_free.restype = None
        L.gp_coarse_free.argtypes = [VP, VP]
        L.gp_partition.restype = ctypes.c_int
        L.gp_partition.argtypes = [ctypes.POINTER(GpGraph), I32, DBL, U64, ctypes.POINTER(GpParams), VP,
                                   ctypes.POINTER(GpResult), VP]
        L.gp_partition_host.restype = ctypes.c_int
        L.gp_partition_host.argtypes = [ctypes.POINTER(GpGraph), I32, DBL, U64, ctypes.POINTER(GpParams), VP,
                                        ctypes.POINTER(GpResult), VP]
        L.gp_mlp_score.restype = ctypes.c_int
        L.gp_mlp_score.argtypes = [ctypes.POINTER(GpGraph), I32, VP, VP, VP, VP]
        L.gp_edge_features.restype = ctypes.c_int
        L.gp_edge_features.argtypes = [ctypes.POINTER(GpGraph), I32, VP, VP]
        L.gp_mlp_train.restype = ctypes.c_int
        L.gp_mlp_train.argtypes = [VP, VP, I64, VP, I32, ctypes.c_float, VP, VP]
        L.gp_mlp_grad.restype = ctypes.c_int
        L.gp_mlp_grad.argtypes = [VP, VP, I64, VP, VP, VP, VP]
        L.gp_mlp_train.argtypes = [VP, VP, I64, VP, I32, ctypes.c_float, VP, VP]
        L.gp_partition_batch.restype = ctypes.c_int
        L.gp_partition_batch.argtypes = [ctypes.POINTER(GpBatchItem), I32, ctypes.POINTER(GpParams),
                                         ctypes.POINTER(GpResult), VP]
        L.gp_lp_set_schedule.restype = ctypes.c_int
        L.gp_lp_set_schedule.argtypes = [ctypes.c_int, ctypes.c_int]
        L.gp_autotune_schedule.restype = ctypes.c_int
        L.gp_autotune_schedule.argtypes = [ctypes.POINTER(GpGraph), VP, VP, VP, VP]
        L.gp_autotune.restype = ctypes.c_int
        L.gp_autotune.argtypes = [ctypes.POINTER(GpGraph), ctypes.POINTER(GpParams), VP, VP]
        L.gp_lp_set_tiles.restype = ctypes.c_int
        L.gp_lp_set_tiles.argtypes = [I64, I64]
        L.gp_lp_set_hub_keep.restype = ctypes.c_int
        L.gp_lp_set_hub_keep.argtypes = [I64, I32]
        L.gp_set_wait_limit.restype = ctypes.c_int
        L.gp_set_wait_limit.argtypes = [U64]
        L.gp_pinned_stage_allocs.restype = I64
        L.gp_pinned_stage_allocs.argtypes = []
        L.gp_free_cached.restype = None
        L.gp_free_cached.argtypes = []
        L.gp_launch_count.restype = I64
        L.gp_launch_count.argtypes = [ctypes.c_int]
        L.gp_profile_enable.restype = ctypes.c_int
        L.gp_profile_enable.argtypes = [ctypes.c_int]
        L.gp_profile_read.restype = ctypes.c_int
        L.gp_profile_read.argtypes = [ctypes.POINTER(GpProfileEntry), ctypes.c_int, ctypes.c_int]
        _lib = L
        _install_torch_allocator(L)
        return L


def _install_torch_allocator(L):
    import torch
    if not torch.cuda.is_available():
        return

    @ALLOC_FN
    def _alloc(nbytes, stream, ctx):
        alloc_calls[0] += 1
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:  # out of memory: report NULL, the library returns GP_ERR_OOM
            return None

    @FREE_FN
    def _free(ptr, nbytes, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    _keep.extend([_alloc, _free])
    L.gp_set_allocator(ctypes.cast(_alloc, VP), ctypes.cast(_free, VP), None)


def free_cached():
    """Returns the device blocks the library keeps for reuse to the allocator."""
    lib().gp_free_cached()


def use_default_allocator():
    """Route the library's temporary memory to cudaMallocAsync instead of PyTorch."""
    lib().gp_set_allocator(None, None, None)


def _check(st: int, where: str):
    if st != GP_OK:
        msg = lib().gp_last_error().decode()
        raise GpError(st, where, msg or lib().gp_status_string(st).decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def version() -> str:
    return lib().gp_version().decode()


def lmax(total_weight: int, k: int, eps: float) -> int:
    return int(lib().gp_lmax(total_weight, k, eps))


def default_params(**overrides) -> GpParams:
    p = GpParams()
    lib().gp_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class DeviceGraph:
    """A graph whose CSR arrays live in device memory (torch tensors)."""

    def __init__(self, n, off, adj, vw=None, ew=None):
        self.n = int(n)
        self.off, self.adj, self.vw, self.ew = off, adj, vw, ew
        self.desc = GpGraph()
        self.desc.n = self.n
        self.desc.m_dir = int(adj.numel())
        self.desc.offsets = off.data_ptr()
        self.desc.adj = adj.data_ptr() if adj.numel() else None
        self.desc.vwgt = vw.data_ptr() if vw is not None else None
        self.desc.ewgt = ew.data_ptr() if ew is not None else None
        import torch
        self.desc.offsets_64 = 1 if off.dtype == torch.int64 else 0
        self.desc.vwgt_64 = 1 if (vw is not None and vw.dtype == torch.int64) else 0
        self.desc.ewgt_64 = 1 if (ew is not None and ew.dtype == torch.int64) else 0

    @property
    def m_dir(self) -> int:
        return int(self.desc.m_dir)

    @classmethod
    def from_host(cls, g, device="cuda", offsets_64: Optional[bool] = None):
        """Copies a ``graphgen.Graph`` to the device. Offsets are int32 when they fit, unless
        ``offsets_64`` forces a width."""
        import torch
        if offsets_64 is None:
            offsets_64 = g.m_dir >= 2**31
        off = torch.from_numpy(np.ascontiguousarray(g.off, dtype=np.int64 if offsets_64 else np.int32)).to(device)
        adj = torch.from_numpy(np.ascontiguousarray(g.adj, dtype=np.int32)).to(device)
        vw = None if g.vw is None else torch.from_numpy(np.ascontiguousarray(g.vw)).to(device)
        ew = None if g.ew is None else torch.from_numpy(np.ascontiguousarray(g.ew)).to(device)
        return cls(g.n, off, adj, vw, ew)

    def to_host(self):
        from graphgen import Graph
        return Graph(self.n, self.off.cpu().numpy().astype(np.int64), self.adj.cpu().numpy(),
                     None if self.vw is None else self.vw.cpu().numpy(),
                     None if self.ew is None else self.ew.cpu().numpy())


def validate(dg: DeviceGraph, stream=None) -> int:
    return int(lib().gp_validate_graph(ctypes.byref(dg.desc), _stream(stream)))


def lp_cluster(dg: DeviceGraph, U: int, rounds: int, seed: int, q=None, stream=None):
    """Size-constrained LP clustering from singletons; returns (labels int32 tensor, stats dict)."""
    import torch
    labels = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.adj.device)
    st = GpLpStats()
    _check(lib().gp_lp_cluster(ctypes.byref(dg.desc), U, rounds, seed, q.data_ptr() if q is not None else None,
                               labels.data_ptr(), ctypes.byref(st), _stream(stream)), "gp_lp_cluster")
    return labels[: dg.n], st.as_dict()


def mls_default_params(**overrides) -> GpMlsParams:
    p = GpMlsParams()
    lib().gp_mls_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def mls(dg: DeviceGraph, part, k: int, lmax_: int, seed: int, params: Optional[GpMlsParams] = None, stream=None):
    """Multi-try k-way local search on a copy of `part`; returns (part, stats dict)."""
    import torch
    part = part.to(torch.int32).clone()
    st = GpMlsStats()
    _check(lib().gp_mls(ctypes.byref(dg.desc), k, lmax_, seed, ctypes.byref(params) if params else None,
                        part.data_ptr(), ctypes.byref(st), _stream(stream)), "gp_mls")
    return part, st.as_dict()


def match(dg: DeviceGraph, U: int, rounds: int, seed: int, stream=None):
    """Matching-based clustering (handshake matching); returns (labels int32 tensor, stats dict)."""
    import torch
    labels = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.adj.device)
    st = GpMatchStats()
    _check(lib().gp_match(ctypes.byref(dg.desc), U, rounds, seed, labels.data_ptr(), ctypes.byref(st),
                          _stream(stream)), "gp_match")
    return labels[: dg.n], st.as_dict()


def lp_cluster_async(dg: DeviceGraph, U: int, rounds: int, seed: int, single_warp: bool = False, stream=None):
    """The paper's asynchronous LP from singletons (non-deterministic unless single_warp)."""
    import torch
    labels = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.adj.device)
    st = GpLpStats()
    _check(lib().gp_lp_cluster_async(ctypes.byref(dg.desc), U, rounds, seed, 1 if single_warp else 0,
                                     labels.data_ptr(), ctypes.byref(st), _stream(stream)), "gp_lp_cluster_async")
    return labels[: dg.n], st.as_dict()


def lp_refine(dg: DeviceGraph, part, k: int, lmax_: int, rounds: int, seed: int, stream=None):
    """LP refinement of a k-way partition in place (a copy is made); returns (part, block weights, stats)."""
    import torch
    part = part.to(torch.int32).clone()
    bw = torch.empty(k, dtype=torch.int64, device=part.device)
    st = GpLpStats()
    _check(lib().gp_lp_refine(ctypes.byref(dg.desc), k, lmax_, rounds, seed, part.data_ptr(), bw.data_ptr(),
                              ctypes.byref(st), _stream(stream)), "gp_lp_refine")
    return part, bw, st.as_dict()


class CoarseGraph:
    """Library-owned coarse graph returned by ``contract``; freed with ``free()`` or on collection."""

    def __init__(self, handle, stream):
        self.handle = handle
        self._stream = stream
        d = lib().gp_coarse_graph(handle).contents
        self.n, self.m_dir = int(d.n), int(d.m_dir)
        self.desc = GpGraph()
        ctypes.pointer(self.desc)[0] = d

    def to_host(self):
        """Copies the coarse CSR to host numpy arrays (int64 offsets and weights)."""
        from graphgen import Graph
        n, m = self.n, self.m_dir
        d = self.desc
        return Graph(n, _wrap(d.offsets, n + 1, "<i8").cpu().numpy(), _wrap(d.adj, m, "<i4").cpu().numpy(),
                     _wrap(d.vwgt, n, "<i8").cpu().numpy(), _wrap(d.ewgt, m, "<i8").cpu().numpy(), "coarse")

    def free(self):
        if self.handle:
            lib().gp_coarse_free(self.handle, self._stream)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _CudaArray:
    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}


def _wrap(ptr, count, typestr):
    """A torch view of library-owned device memory (no copy)."""
    import torch
    if count == 0 or not ptr:
        return torch.empty(0, dtype={"<i8": torch.int64, "<i4": torch.int32}[typestr], device="cuda")
    return torch.as_tensor(_CudaArray(ptr, count, typestr), device="cuda")


def contract(dg: DeviceGraph, labels, stream=None):
    """Contraction of a clustering; returns (CoarseGraph, f2c int32 tensor)."""
    import torch
    f2c = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.adj.device)
    h = VP()
    s = _stream(stream)
    _check(lib().gp_contract(ctypes.byref(dg.desc), labels.data_ptr(), ctypes.byref(h), f2c.data_ptr(), s),
           "gp_contract")
    return CoarseGraph(h, s), f2c[: dg.n]


@dataclass
class PartitionResult:
    cut: int
    max_block_weight: int
    lmax: int
    imbalanced: int
    levels: int
    best_try: int
    n_isolated: int
    level_n: list
    level_m: list
    try_cut: list
    try_imbalanced: list
    lp_edges: int
    lp_moves: int
    plain_cut: int
    learned_cut: int
    ms_total: float
    ms_coarsen: float
    ms_initial: float
    ms_refine: float


def _result(r: GpResult, tries: int) -> PartitionResult:
    return PartitionResult(r.cut, r.max_block_weight, r.lmax, r.imbalanced, r.levels, r.best_try, r.n_isolated,
                           list(r.level_n[: r.levels + 1]), list(r.level_m[: r.levels + 1]),
                           list(r.try_cut[:tries]), list(r.try_imbalanced[:tries]), r.lp_edges, r.lp_moves,
                           r.plain_cut, r.learned_cut, r.ms_total, r.ms_coarsen, r.ms_initial, r.ms_refine)


def partition(dg: DeviceGraph, k: int, eps: float, seed: int, params: Optional[GpParams] = None, stream=None,
              out=None):
    """Full multilevel partition; returns (part int32 tensor, PartitionResult)."""
    import torch
    part = out if out is not None else torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.adj.device)
    res = GpResult()
    _check(lib().gp_partition(ctypes.byref(dg.desc), k, eps, seed, ctypes.byref(params) if params else None,
                              part.data_ptr(), ctypes.byref(res), _stream(stream)), "gp_partition")
    tries = params.ip_tries if params else 4
    return part[: dg.n], _result(res, tries)


class HostGraph:
    """Host CSR (numpy, optionally pinned torch tensors) described for gp_partition_host."""

    def __init__(self, g, pin: bool = True):
        import torch
        self.n = g.n
        arrs = {"off": np.ascontiguousarray(g.off, dtype=np.int64 if g.m_dir >= 2**31 else np.int32),
                "adj": np.ascontiguousarray(g.adj, dtype=np.int32)}
        if g.vw is not None:
            arrs["vw"] = np.ascontiguousarray(g.vw)
        if g.ew is not None:
            arrs["ew"] = np.ascontiguousarray(g.ew)
        self.t = {}
        for k, a in arrs.items():
            t = torch.from_numpy(a)
            self.t[k] = t.pin_memory() if pin else t
        self.part = torch.empty(max(g.n, 1), dtype=torch.int32)
        if pin:
            self.part = self.part.pin_memory()
        self.desc = GpGraph()
        self.desc.n = g.n
        self.desc.m_dir = g.m_dir
        self.desc.offsets = self.t["off"].data_ptr()
        self.desc.adj = self.t["adj"].data_ptr() if g.m_dir else None
        self.desc.vwgt = self.t["vw"].data_ptr() if "vw" in self.t else None
        self.desc.ewgt = self.t["ew"].data_ptr() if "ew" in self.t else None
        self.desc.offsets_64 = 1 if self.t["off"].dtype == torch.int64 else 0
        self.desc.vwgt_64 = 1 if ("vw" in self.t and self.t["vw"].dtype == torch.int64) else 0
        self.desc.ewgt_64 = 1 if ("ew" in self.t and self.t["ew"].dtype == torch.int64) else 0
        self.h2d_bytes = sum(int(t.numel() * t.element_size()) for t in self.t.values())
        self.d2h_bytes = 4 * g.n


def partition_host(hg: HostGraph, k: int, eps: float, seed: int, params: Optional[GpParams] = None, stream=None):
    """gp_partition on host buffers (the call copies in and out); returns (part numpy view, result)."""
    res = GpResult()
    _check(lib().gp_partition_host(ctypes.byref(hg.desc), k, eps, seed, ctypes.byref(params) if params else None,
                                   hg.part.data_ptr(), ctypes.byref(res), _stream(stream)), "gp_partition_host")
    tries = params.ip_tries if params else 4
    return hg.part[: hg.n].numpy(), _result(res, tries)


def lp_set_schedule(deg_warp: int = 0, deg_cta: int = 0):
    """Degree-bin thresholds of the LP kernels for gp_lp_cluster/gp_lp_refine (0 = defaults)."""
    _check(lib().gp_lp_set_schedule(deg_warp, deg_cta), "gp_lp_set_schedule")


def lp_set_tiles(hub_batch_slots: int = 0, verts_per_block: int = 0):
    """LP tile sizes for gp_lp_cluster/gp_lp_refine (0 = defaults); results never depend on them."""
    _check(lib().gp_lp_set_tiles(hub_batch_slots, verts_per_block), "gp_lp_set_tiles")


def lp_set_hub_keep(slots: int = 0, max_load_pct: int = 0):
    """Kept hub tables: slots for gp_lp_cluster/gp_lp_refine (0 = default budget, negative = never
    kept); max_load_pct for every LP call (0 = default 75; 1 = stale at the first new label)."""
    _check(lib().gp_lp_set_hub_keep(slots, max_load_pct), "gp_lp_set_hub_keep")


def set_wait_limit(ns: int = 0):
    """Limit of every bounded device wait in nanoseconds (0 = the default of 20 s)."""
    _check(lib().gp_set_wait_limit(ns), "gp_set_wait_limit")


def pinned_stage_allocs() -> int:
    """Pinned host staging buffers the library has allocated since load."""
    return int(lib().gp_pinned_stage_allocs())


def launch_count(reset: bool = False) -> int:
    """Kernel launches issued by the library (optionally resetting the counter)."""
    return int(lib().gp_launch_count(1 if reset else 0))


def profile_enable(on: bool = True):
    lib().gp_profile_enable(1 if on else 0)


def profile_read(reset: bool = False) -> list:
    buf = (GpProfileEntry * 64)()
    n = lib().gp_profile_read(buf, 64, 1 if reset else 0)
    return [{"name": buf[i].name.decode(), "launches": buf[i].launches, "ms": buf[i].ms, "items": buf[i].items,
             "edges": buf[i].edges, "bytes": buf[i].bytes} for i in range(n)]


# ---------------------------------------------------------------------------------------------- learned
MLP_BYTES = 256 * 2 + 32 * 2 + 32 * 4 + 4 + 7 * 4  # sizeof(gp_mlp)


def _bf16_bits(a) -> np.ndarray:
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def bf16_round(a) -> np.ndarray:
    """Values of `a` rounded to bfloat16 (round to nearest even), as float64."""
    bits = _bf16_bits(a).astype(np.uint32) << 16
    return bits.view(np.float32).astype(np.float64)


def mlp_pack(w1, b1, w2, b2, device="cuda"):
    """A device gp_mlp (uint8 tensor): w1 [32,8] and w2 [32] rounded to bfloat16, biases float32."""
    import torch
    buf = np.zeros(MLP_BYTES, dtype=np.uint8)
    buf[0:512] = _bf16_bits(np.asarray(w1, dtype=np.float32).reshape(256)).view(np.uint8)
    buf[512:576] = _bf16_bits(np.asarray(w2, dtype=np.float32).reshape(32)).view(np.uint8)
    buf[576:704] = np.asarray(b1, dtype=np.float32).reshape(32).view(np.uint8)
    buf[704:708] = np.asarray([b2], dtype=np.float32).view(np.uint8)
    return torch.from_numpy(buf).to(device)


def mlp_unpack(t):
    """(w1 [32,8], b1 [32], w2 [32], b2) as float64 from a device gp_mlp."""
    buf = t.cpu().numpy()
    w1 = (buf[0:512].view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64).reshape(32, 8)
    w2 = (buf[512:576].view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    b1 = buf[576:704].view(np.float32).astype(np.float64)
    b2 = float(buf[704:708].view(np.float32)[0])
    return w1, b1, w2, b2


def edge_features(dg: DeviceGraph, level: int, stream=None):
    """Per-entry features [m_dir, 8] (float32, device)."""
    import torch
    out = torch.empty((max(dg.m_dir, 1), 8), dtype=torch.float32, device=dg.adj.device)
    _check(lib().gp_edge_features(ctypes.byref(dg.desc), level, out.data_ptr(), _stream(stream)), "gp_edge_features")
    return out[: dg.m_dir]


def mlp_score(dg: DeviceGraph, level: int, mlp, stream=None):
    """Scores s (float32) and q = round-half-even(s * 2^15) (int32) of every CSR entry."""
    import torch
    s = torch.empty(max(dg.m_dir, 1), dtype=torch.float32, device=dg.adj.device)
    q = torch.empty(max(dg.m_dir, 1), dtype=torch.int32, device=dg.adj.device)
    _check(lib().gp_mlp_score(ctypes.byref(dg.desc), level, mlp.data_ptr(), s.data_ptr(), q.data_ptr(),
                              _stream(stream)), "gp_mlp_score")
    return s[: dg.m_dir], q[: dg.m_dir]


def mlp_train(feat, y, mlp, steps: int, lr: float, stream=None) -> np.ndarray:
    """Full-batch Adam on (feat [m,8] float32, y [m] float32), updating `mlp` in place; returns the loss
    before each step."""
    losses = np.zeros(steps, dtype=np.float32)
    _check(lib().gp_mlp_train(feat.data_ptr(), y.data_ptr(), int(feat.shape[0]), mlp.data_ptr(), steps, lr,
                              losses.ctypes.data, _stream(stream)), "gp_mlp_train")
    return losses


def mlp_grad(feat, y, mlp, stream=None):
    """(mean loss, gradient [321] = dW1 (row-major), db1, dW2, db2) in FP32 from the bf16 weights."""
    loss = ctypes.c_float(0)
    grad = np.zeros(321, dtype=np.float32)
    _check(lib().gp_mlp_grad(feat.data_ptr(), y.data_ptr(), int(feat.shape[0]), mlp.data_ptr(), ctypes.byref(loss),
                             grad.ctypes.data, _stream(stream)), "gp_mlp_grad")
    return float(loss.value), grad


# ---------------------------------------------------------------------------------------------- batch
def partition_batch(graphs, ks, eps, seeds, params: Optional[GpParams] = None, stream=None):
    """Partitions several DeviceGraphs in one call; returns (list of part tensors, list of results)."""
    import torch
    n = len(graphs)
    items = (GpBatchItem * max(n, 1))()
    parts = []
    for i, dg in enumerate(graphs):
        part = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.adj.device)
        parts.append(part)
        items[i].g = dg.desc
        items[i].k = int(ks[i])
        items[i].eps = float(eps[i] if hasattr(eps, "__len__") else eps)
        items[i].seed = int(seeds[i])
        items[i].part_out = part.data_ptr()
    res = (GpResult * max(n, 1))()
    _check(lib().gp_partition_batch(items, n, ctypes.byref(params) if params else None, res, _stream(stream)),
           "gp_partition_batch")
    tries = params.ip_tries if params else 4
    return [parts[i][: graphs[i].n] for i in range(n)], [_result(res[i], tries) for i in range(n)]


def autotune(dg: DeviceGraph, params: Optional[GpParams] = None, stream=None):
    """Degree bins and tile sizes picked by timing LP rounds of dg; returns (params, ms)."""
    p = params if params is not None else default_params()
    ms = ctypes.c_double(0)
    _check(lib().gp_autotune(ctypes.byref(dg.desc), ctypes.byref(p), ctypes.byref(ms), _stream(stream)),
           "gp_autotune")
    return p, float(ms.value)


def autotune_schedule(dg: DeviceGraph, stream=None):
    """(deg_warp, deg_cta, ms) picked by timing LP rounds of dg under the candidate schedules."""
    w, c, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0)
    _check(lib().gp_autotune_schedule(ctypes.byref(dg.desc), ctypes.byref(w), ctypes.byref(c), ctypes.byref(ms),
                                      _stream(stream)), "gp_autotune_schedule")
    return int(w.value), int(c.value), float(ms.value)
