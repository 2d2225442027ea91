"""Host-side checks of the uneven-batch plan (no GPU): request validation and
plan bookkeeping."""
import numpy as np
import pytest

import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import workloads as W


def test_plan_validation():
    ok = cf.requests([0, 1, 2], [4, 8, 16], [0, 4, 12], [0, 0, 0])
    for prec in (cf.FP64, cf.FP32_COMP):
        h = cf.chessfad_ragged_plan_create(ok, prec)
        info = cf.chessfad_ragged_plan_info(h)
        assert info["ntiles"] == 3 and info["workspace_bytes"] > 0 and info["smem_bytes"] > 0
        assert cf.chessfad_ragged_plan_destroy(h) == 0
    lib = cf.load()
    import ctypes
    h = ctypes.c_void_p()
    for fns, ns, offs, eoffs, code in (([3], [4], [0], [0], -1), ([0], [0], [0], [0], -2), ([0], [513], [0], [0], -2),
                                       ([0], [4], [-1], [0], -11), ([2], [4], [0], [-5], -11)):
        r = cf.requests(fns, ns, offs, eoffs)
        assert lib.chessfad_ragged_plan_create(r.ctypes.data, 1, 1, 0, ctypes.byref(h)) == code
    r = cf.requests([0], [4], [0])
    assert lib.chessfad_ragged_plan_create(r.ctypes.data, 1, 5, 0, ctypes.byref(h)) == -7
    assert lib.chessfad_ragged_plan_create(r.ctypes.data, 1, 1, 4, ctypes.byref(h)) == -4
    assert lib.chessfad_ragged_plan_create(None, 3, 1, 0, ctypes.byref(h)) == -5
    assert lib.chessfad_ragged_plan_create(None, 0, 1, 0, ctypes.byref(h)) == 0
    assert cf.chessfad_ragged_plan_info(h.value)["ntiles"] == 0
    cf.chessfad_ragged_plan_destroy(h.value)
    # run-time argument checks happen before any CUDA call
    h = cf.chessfad_ragged_plan_create(cf.requests([2], [4], [0], [0]))
    ws = cf.chessfad_ragged_plan_info(h)["workspace_bytes"]
    assert lib.chessfad_hvp_ragged(h, 16, 16, 16, None, 16, ws, None) == -6
    assert lib.chessfad_hvp_ragged(h, 16, 16, 16, None, 16, ws - 1, None) == -8
    assert lib.chessfad_hvp_ragged(h, 16, 16, 16, None, None, ws, None) == -8
    assert lib.chessfad_hvp_ragged(None, 16, 16, 16, None, 16, ws, None) == -11
    cf.chessfad_ragged_plan_destroy(h)


def test_plan_tiles_cover_the_uneven_batch():
    rg = W.make_ragged(nreq=2000, seed=4)
    r = cf.requests(rg.fns, rg.ns, rg.offs, rg.eoffs)
    h = cf.chessfad_ragged_plan_create(r, cf.FP32_COMP, 8)
    info = cf.chessfad_ragged_plan_info(h)
    groups = {}
    for f, n in zip(rg.fns, rg.ns):
        groups[(int(f), int(n))] = groups.get((int(f), int(n)), 0) + 1
    # every group contributes at least one tile; a tile holds at most 256 rows
    assert info["ntiles"] >= len(groups)
    assert info["ntiles"] >= sum(-(-cnt * n // 256) for (f, n), cnt in groups.items())
    assert info["smem_bytes"] <= 227 * 1024
    cf.chessfad_ragged_plan_destroy(h)
