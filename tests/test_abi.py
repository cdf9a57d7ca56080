"""The C-ABI library builds, loads and exports every function that include/gpart.h declares.

No compute call is made here (these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gpart.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for want in ["gp_lp_cluster", "gp_contract", "gp_lp_refine", "gp_partition", "gp_partition_host",
                 "gp_mlp_score", "gp_mlp_train", "gp_partition_batch"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_1710_08231_gb300 as gp
    path = gp.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    import paper_1710_08231_gb300 as gp
    gp.build()
    lib = ctypes.CDLL(gp.LIB_PATH)
    lib.gp_lmax.restype = ctypes.c_int64
    lib.gp_lmax.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double]
    assert lib.gp_lmax(65536, 2, 0.03) == 33751
    assert lib.gp_lmax(1048576, 16, 0.03) == 67502
    lib.gp_status_string.restype = ctypes.c_char_p
    assert lib.gp_status_string(0) == b"ok"
    p = gp.GpParams()
    lib.gp_default_params(ctypes.byref(p))
    assert (p.rounds_coarsen, p.rounds_refine, p.ip_tries, p.cluster_div) == (10, 25, 4, 14)


def test_host_setters_validate_and_restore():
    """Process-wide LP settings are host state: out-of-range values are refused, 0 restores a default."""
    import paper_1710_08231_gb300 as gp
    gp.build()
    L = gp.lib()
    assert L.gp_lp_set_hub_keep(0, 96) == gp.GP_ERR_INVALID_ARG
    assert L.gp_lp_set_hub_keep(0, -1) == gp.GP_ERR_INVALID_ARG
    assert L.gp_lp_set_hub_keep(-1, 1) == 0 and L.gp_lp_set_hub_keep(0, 0) == 0
    assert L.gp_lp_set_tiles(-1, 0) == gp.GP_ERR_INVALID_ARG
    assert L.gp_lp_set_tiles(4096, 16) == 0 and L.gp_lp_set_tiles(0, 0) == 0
    assert L.gp_lp_set_schedule(-1, 0) == gp.GP_ERR_INVALID_ARG and L.gp_lp_set_schedule(0, 0) == 0
    p = gp.GpParams()
    L.gp_default_params(ctypes.byref(p))
    assert (p.hub_batch_slots, p.verts_per_block, p.hub_keep_slots) == (0, 0, 0)  # defaults chosen by the library
