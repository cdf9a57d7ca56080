"""Failure detection without a GPU fault.

* A bounded device wait that runs out: the wait limit of the LP kernel's grid barriers is set to one
  nanosecond, so the first barrier at which blocks arrive apart gives up. The call must return
  GP_ERR_TIMEOUT (every CTA returned, the context stays usable) and, with the default limit restored,
  the next call must give the labels it gave before.
* An allocator that fails: the installed allocator callback returns NULL after a number of successful
  calls. Every call must return GP_ERR_OOM, give every block it obtained back (none is leaked), and
  the library must work again once a working allocator is installed.
"""
import ctypes

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
    m.lp_set_tiles(0, 0)
    m.lp_set_hub_keep(0, 0)
    return m


def test_barrier_wait_runs_out(gp):
    g = gg.rgg(200_000, 12.0, 4)  # about 3,000 blocks' worth of vertices: a many-block problem
    dg = gp.DeviceGraph.from_host(g)
    ref, st_ref = gp.lp_cluster(dg, 60, 10, 3)
    ref = ref.cpu().numpy()
    gp.set_wait_limit(1)
    try:
        with pytest.raises(gp.GpError) as ei:
            gp.lp_cluster(dg, 60, 10, 3)
        assert ei.value.status == gp.GP_ERR_TIMEOUT
        assert "barrier" in str(ei.value)
    finally:
        gp.set_wait_limit(0)
    lab, st = gp.lp_cluster(dg, 60, 10, 3)
    assert np.array_equal(lab.cpu().numpy(), ref) and st == st_ref
    lab_o, _, _ = O.lp_cluster(g, 60, 10, 3)
    assert np.array_equal(ref, lab_o)


class _FailingAllocator:
    """Allocator callback backed by PyTorch's caching allocator that fails after `budget` calls and
    tracks the blocks outstanding."""

    def __init__(self, budget):
        import torch
        self.budget = budget
        self.calls = 0
        self.live = {}

        @gp_alloc_fn
        def alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls > self.budget:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
            self.live[p] = int(nbytes)
            return p

        @gp_free_fn
        def free(ptr, nbytes, stream, ctx):
            if ptr:
                assert self.live.pop(ptr) == int(nbytes)
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc, self.free = alloc, free


gp_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
gp_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


def _install(gp, fa):
    gp.lib().gp_set_allocator(ctypes.cast(fa.alloc, ctypes.c_void_p), ctypes.cast(fa.free, ctypes.c_void_p), None)


def test_allocator_failure_returns_oom_without_leak(gp):
    g = gg.rmat(13, 8, seed=2)
    dg = gp.DeviceGraph.from_host(g)
    ref_part, ref_res = gp.partition(dg, 8, 0.03, 1)
    ref_part = ref_part.cpu().numpy()
    L = gp.lib()
    import torch
    # the number of allocator calls one partition makes with an empty block cache
    counting = _FailingAllocator(10**9)
    _install(gp, counting)
    try:
        part, res = gp.partition(dg, 8, 0.03, 1)
        assert np.array_equal(part.cpu().numpy(), ref_part)
        need = counting.calls
        assert need >= 1
        # every allocation point in turn fails
        for budget in range(need):
            fa = _FailingAllocator(budget)
            _install(gp, fa)  # (returns the previous allocator's cached blocks to it)
            with pytest.raises(gp.GpError) as ei:
                gp.partition(dg, 8, 0.03, 1)
            assert ei.value.status == gp.GP_ERR_OOM, (budget, ei.value)
            torch.cuda.synchronize()
            L.gp_free_cached()  # blocks kept for reuse go back to this allocator
            assert fa.calls >= budget + 1
            assert not fa.live, f"budget {budget}: {len(fa.live)} blocks leaked"
        torch.cuda.synchronize()
        L.gp_free_cached()
        assert not counting.live
    finally:
        gp._install_torch_allocator(L)
    part, res = gp.partition(dg, 8, 0.03, 1)
    assert np.array_equal(part.cpu().numpy(), ref_part) and res.cut == ref_res.cut
