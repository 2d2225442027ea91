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


def _sym_rows(n, csize):
    """Rows per symmetric tile: lanes per row doubled from the plain choice
    until a tile holds no more rows than the request has."""
    nch = -(-n // csize)
    tpr = 1
    while tpr * 2 <= max(1, nch // 8):
        tpr *= 2
    tpr = min(32, tpr)
    while tpr < 32 and 256 // tpr > n:
        tpr *= 2
    return 256 // tpr


@pytest.mark.parametrize("csize", [8, 16])
def test_symmetric_tiles_and_accumulator_workspace(csize):
    """Fletcher-Powell requests with n >= 128 get tiles of one point each
    (ceil(n / rows) of them) and n FP64 accumulators plus a row counter in the
    workspace; smaller requests and other functions keep the plain tiling."""
    big = [(2, 128), (2, 200), (2, 512), (2, 300)]
    fns = [f for f, _ in big]
    ns = [n for _, n in big]
    offs = np.concatenate([[0], np.cumsum(ns[:-1])])
    h = cf.chessfad_ragged_plan_create(cf.requests(fns, ns, offs, [0] * len(ns)), cf.FP32_COMP, csize)
    info = cf.chessfad_ragged_plan_info(h)
    assert info["ntiles"] == sum(-(-n // _sym_rows(n, csize)) for n in ns)
    assert info["workspace_bytes"] >= 8 * sum(ns) + 4 * len(ns)
    cf.chessfad_ragged_plan_destroy(h)
    # the same sizes as Rosenbrock requests: plain tiles, no accumulators
    h2 = cf.chessfad_ragged_plan_create(cf.requests([0] * len(ns), ns, offs), cf.FP32_COMP, csize)
    info2 = cf.chessfad_ragged_plan_info(h2)
    assert info2["workspace_bytes"] < info["workspace_bytes"]
    cf.chessfad_ragged_plan_destroy(h2)
    # one request below the threshold: plain tiling of a 127-variable request
    h3 = cf.chessfad_ragged_plan_create(cf.requests([2], [127], [0], [0]), cf.FP32_COMP, csize)
    assert cf.chessfad_ragged_plan_info(h3)["ntiles"] == 1
    cf.chessfad_ragged_plan_destroy(h3)
