"""gp_lp_cluster_noalloc: label-propagation clustering for callers that cannot allocate device memory.

Such callers (code that may not call cudaMalloc or a caching allocator while it runs) get the same
clustering as gp_lp_cluster, computed with a fixed scratch array inside the library. These tests call
both entry points through the C ABI on the same inputs and require identical labels and counters on
two calls in a row, and check that the allocation-free call never asks the installed allocator for
memory. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import graphgen as gg

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


def _noalloc(gp, dg, U, rounds, seed, q=None):
    import torch
    labels = torch.full((dg.n,), -1, dtype=torch.int32, device="cuda")
    st = gp.GpLpStats()
    rc = gp.lib().gp_lp_cluster_noalloc(ctypes.byref(dg.desc), U, rounds, seed,
                                        q.data_ptr() if q is not None else None, labels.data_ptr(),
                                        ctypes.byref(st), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == gp.GP_OK, gp.lib().gp_last_error().decode()
    return labels.cpu().numpy(), st.as_dict()


CASES = [
    ("rgg10k", lambda: gg.rgg(10000, 12.0, 3), 0, 0),
    ("rmat12_hub_tables", lambda: gg.rmat(12, 8, seed=5), 32, 32),
    ("rmat11_weighted", lambda: gg.rmat(11, 8, seed=6, weighted=True), 0, 0),
]


@pytest.mark.parametrize("name,make,dw,dc", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_entry_point(gp, name, make, dw, dc):
    g = make()
    dg = gp.DeviceGraph.from_host(g)
    gp.lp_set_schedule(dw, dc)
    try:
        ref, st_ref = gp.lp_cluster(dg, 50, 10, 77)
        ref = ref.cpu().numpy()
        for _ in range(2):  # two calls in a row share (and reuse) the fixed scratch array
            before = gp.alloc_calls[0]
            lab, st = _noalloc(gp, dg, 50, 10, 77)
            assert gp.alloc_calls[0] == before, "the allocation-free call requested device memory"
            assert np.array_equal(lab, ref)
            assert st == st_ref
    finally:
        gp.lp_set_schedule(0, 0)


def test_noalloc_rejects_graphs_beyond_the_limit(gp):
    g = gg.grid(200, 200)  # 40,000 vertices > 32,768
    dg = gp.DeviceGraph.from_host(g)
    import torch
    labels = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = gp.GpLpStats()
    rc = gp.lib().gp_lp_cluster_noalloc(ctypes.byref(dg.desc), 50, 10, 1, None, labels.data_ptr(),
                                        ctypes.byref(st), None)
    assert rc == gp.GP_ERR_UNSUPPORTED
    assert "32768" in gp.lib().gp_last_error().decode()


def test_noalloc_makes_no_pinned_host_allocation_on_a_new_thread(gp):
    """A thread's first call would have to allocate the pinned staging buffer of the library's
    read-backs; the allocation-free call must not: its counters go straight to ordinary host memory."""
    import threading
    g = gg.rgg(8000, 12.0, 9)
    dg = gp.DeviceGraph.from_host(g)
    ref, st_ref = gp.lp_cluster(dg, 40, 10, 5)
    ref = ref.cpu().numpy()
    out = {}

    def run():
        import torch
        torch.cuda.set_device(0)
        before = gp.pinned_stage_allocs()
        out["res"] = [_noalloc(gp, dg, 40, 10, 5) for _ in range(2)]
        out["pinned"] = gp.pinned_stage_allocs() - before

    t = threading.Thread(target=run)
    t.start()
    t.join()
    assert out["pinned"] == 0
    for lab, st in out["res"]:
        assert np.array_equal(lab, ref) and st == st_ref
