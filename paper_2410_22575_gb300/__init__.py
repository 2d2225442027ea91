"""GB300-native chunked-hDual Hessian / Hessian-vector-product library.

A thin ctypes binding over ``_build/libchessfad.so`` (see ``include/chessfad.h``
for the C ABI).  The functions named ``chessfad_*`` have the C names and take
the C arguments; device buffers may be passed as ``torch`` CUDA tensors (their
``data_ptr()`` is used) or as raw integer addresses, streams as
``torch.cuda.Stream`` or raw handles.  PyTorch is only the allocator and stream
provider: every step of the hot path runs in the library's CUDA kernels.  There
is no CPU fallback -- if the library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

ROSENBROCK, ACKLEY, FLETCHER_POWELL = 0, 1, 2
FP64, FP32_COMP = 0, 1
MAX_N = 512

SUCCESS = 0
ERR = {
    -1: "FUNCTION", -2: "SIZE", -3: "BATCH", -4: "CHUNK", -5: "NULL", -6: "PARAMS",
    -7: "PRECISION", -8: "WORKSPACE", -9: "CONFIG", -10: "CUDA", -11: "PLAN",
}

_lock = threading.Lock()
_lib = None


class ChessfadError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else f"{strerror(status)} ({status})")


class FPParams(ctypes.Structure):
    """chessfad_fp_params: device pointers to A, B (row-major, leading dim ld) and E."""
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("E", ctypes.c_void_p), ("ld", ctypes.c_int)]


PLAIN, SYMMETRIC, SYMMETRIC_SPARSE, POINT = 0, 1, 2, 3


class Config(ctypes.Structure):
    """chessfad_config: chunk size, threads per row, CTA size (plain method),
    method, threads per point (symmetric method); 0 = default."""
    _fields_ = [("csize", ctypes.c_int), ("threads_per_row", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("method", ctypes.c_int), ("threads_per_point", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"csize": self.csize, "threads_per_row": self.threads_per_row, "block_threads": self.block_threads,
                "method": {PLAIN: "plain", SYMMETRIC: "symmetric", SYMMETRIC_SPARSE: "symmetric_sparse",
                           POINT: "point"}.get(
                    self.method, str(self.method)),
                "threads_per_point": self.threads_per_point}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libchessfad not built ({_build.LIB}); run python -m paper_2410_22575_gb300.build")
        lib = ctypes.CDLL(_build.LIB)
        P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
        lib.chessfad_hvp.argtypes = [I, I, L, I, P, P, P, P, I, P]
        lib.chessfad_hessian.argtypes = [I, I, L, I, P, P, P, I, P]
        lib.chessfad_hvp_config.argtypes = [I, I, L, P, P, P, P, P, I, P]
        lib.chessfad_hessian_config.argtypes = [I, I, L, P, P, P, P, I, P]
        lib.chessfad_default_config.argtypes = [I, I, L, I, P]
        lib.chessfad_resolve_config.argtypes = [I, I, L, I, I, P, P]
        lib.chessfad_autotune_hessian.argtypes = [I, I, L, P, P, P, I, P, P]
        lib.chessfad_autotune_hvp.argtypes = [I, I, L, P, P, P, P, I, P, P]
        lib.chessfad_peak_flops.argtypes = [I, ctypes.POINTER(ctypes.c_double)]
        lib.chessfad_peak_info.argtypes = [I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.chessfad_peak_operand_rates.argtypes = [I, ctypes.POINTER(ctypes.c_double),
                                                    ctypes.POINTER(ctypes.c_double)]
        lib.chessfad_kernel_info.argtypes = [I, I, I, I, ctypes.POINTER(I), ctypes.POINTER(L)]
        lib.chessfad_eft.argtypes = [P, P, L, P, P, P, P, P]
        lib.chessfad_eft.restype = I
        lib.chessfad_compensated_rows.argtypes = [P, P, L, I, I, I, P, P]
        lib.chessfad_compensated_rows.restype = I
        lib.chessfad_ragged_plan_create.argtypes = [P, L, I, I, ctypes.POINTER(P)]
        lib.chessfad_ragged_plan_destroy.argtypes = [P]
        lib.chessfad_ragged_plan_info.argtypes = [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(L),
                                                  ctypes.POINTER(ctypes.c_size_t)]
        lib.chessfad_ragged_plan_upload.argtypes = [P, P, ctypes.c_size_t, P]
        lib.chessfad_ragged_plan_group_config.argtypes = [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I),
                                                          ctypes.POINTER(I)]
        lib.chessfad_ragged_autotune.argtypes = [P, L, I, P, P, P, P, P, ctypes.c_size_t, P, ctypes.POINTER(L)]
        lib.chessfad_ragged_tuned_config.argtypes = [I, I, I, ctypes.POINTER(I), ctypes.POINTER(I),
                                                     ctypes.POINTER(I)]
        lib.chessfad_hvp_ragged.argtypes = [P, P, P, P, P, P, ctypes.c_size_t, P]
        lib.chessfad_hvp_ragged_noalloc.argtypes = [P, P, P, P, P, P]
        lib.chessfad_hvp_ragged_noalloc.restype = I
        lib.chessfad_user_fn_create.argtypes = [ctypes.c_char_p, ctypes.c_char_p, I, I, ctypes.POINTER(P),
                                                ctypes.c_char_p, ctypes.c_size_t]
        lib.chessfad_user_fn_destroy.argtypes = [P]
        lib.chessfad_user_fn_info.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                              ctypes.POINTER(I)]
        lib.chessfad_user_hvp.argtypes = [P, I, L, P, P, P, P, P]
        lib.chessfad_user_hessian.argtypes = [P, I, L, P, P, P, P]
        lib.chessfad_user_hvp_config.argtypes = [P, I, L, P, P, P, P, P, P]
        lib.chessfad_user_hessian_config.argtypes = [P, I, L, P, P, P, P, P]
        for name in ("chessfad_user_fn_create", "chessfad_user_fn_destroy", "chessfad_user_fn_info",
                     "chessfad_user_hvp", "chessfad_user_hessian", "chessfad_user_hvp_config",
                     "chessfad_user_hessian_config"):
            getattr(lib, name).restype = I
        lib.chessfad_hvp_host.argtypes = [I, I, L, I, P, P, P, P, P, P, P, I, I, P]
        lib.chessfad_hvp_host.restype = I
        lib.chessfad_strerror.argtypes = [I]
        lib.chessfad_strerror.restype = ctypes.c_char_p
        lib.chessfad_version.argtypes = []
        for name in ("chessfad_hvp", "chessfad_hessian", "chessfad_hvp_config", "chessfad_hessian_config",
                     "chessfad_default_config", "chessfad_resolve_config", "chessfad_autotune_hvp",
                     "chessfad_autotune_hessian", "chessfad_peak_flops",
                     "chessfad_peak_info", "chessfad_peak_operand_rates",
                     "chessfad_kernel_info", "chessfad_version", "chessfad_ragged_plan_create",
                     "chessfad_ragged_plan_destroy", "chessfad_ragged_plan_info", "chessfad_ragged_plan_upload",
                     "chessfad_hvp_ragged", "chessfad_ragged_plan_group_config", "chessfad_ragged_autotune",
                     "chessfad_ragged_tuned_config"):
            getattr(lib, name).restype = I
        _lib = lib
        return lib


def _addr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    raise TypeError(f"expected a device tensor or an address, got {type(t)}")


def _stream(s) -> int | None:
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _require(t, name, dtype, shape=None):
    """Check a tensor argument of the conveniences below before anything is
    launched: a torch tensor of `shape` (when given) and `dtype`, contiguous
    (row-major).  The C-named calls take raw addresses and cannot check any
    of this."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype} for this precision, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous (row-major) tensor")


def _require_cuda(**tensors):
    """Every given tensor lives on one CUDA device (checked after _require, so
    a misshapen argument is named first).  None entries are skipped."""
    first = None
    for name, t in tensors.items():
        if t is None:
            continue
        if t.device.type != "cuda" or (first is not None and t.device != first):
            raise ValueError(f"{name}: expected a tensor on {first or 'a CUDA device'}, got {t.device}")
        if first is None:
            first = t.device


def _points(x, name="x"):
    """(batch, n) of a [batch, n] tensor."""
    import torch

    if not isinstance(x, torch.Tensor) or x.dim() != 2:
        raise ValueError(f"{name}: expected a [batch, n] torch tensor")
    return int(x.shape[0]), int(x.shape[1])


def fp_params(A, B, E) -> FPParams:
    """FPParams from device tensors: A, B float64 row-major [rows, ld] (the
    leading n x n block is used), E float64 [>= n]."""
    import torch

    if not isinstance(A, torch.Tensor) or A.dim() != 2:
        raise ValueError("A: expected a [rows, ld] torch tensor")
    _require(A, "A", torch.float64)
    _require(B, "B", torch.float64, A.shape)
    if not isinstance(E, torch.Tensor) or E.dim() != 1:
        raise ValueError("E: expected a 1-D torch tensor")
    _require(E, "E", torch.float64)
    _require_cuda(A=A, B=B, E=E)
    p = FPParams(_addr(A), _addr(B), _addr(E), int(A.shape[1]))
    p._extent = (int(A.shape[0]), int(A.shape[1]), int(E.numel()))  # rows, ld, entries of E
    return p


def _require_fp_extent(fn, n, params):
    """The Fletcher-Powell parameters cover n variables (rows and E entries;
    the library checks ld itself)."""
    extent = getattr(params, "_extent", None) if params is not None else None
    if fn == FLETCHER_POWELL and extent is not None and (extent[0] < n or extent[2] < n):
        raise ValueError(f"Fletcher-Powell parameters hold {extent[0]} rows and {extent[2]} E entries, "
                         f"fewer than n = {n}")


def _check(status: int, what: str) -> int:
    if status != SUCCESS:
        raise ChessfadError(status, what)
    return status


def strerror(status: int) -> str:
    return load().chessfad_strerror(status).decode()


# ------------------------------------------------------------ C-named calls
def chessfad_hvp(fn, n, batch, csize, x, v, out, params=None, prec=FP64, stream=None) -> int:
    p = ctypes.byref(params) if params is not None else None
    return load().chessfad_hvp(fn, n, batch, csize, _addr(x), _addr(v), _addr(out), p, prec, _stream(stream))


def chessfad_hvp_host(fn, n, batch, csize, x_host, v_host, out_host, x_dev, v_dev, out_dev, params=None,
                      prec=FP64, slices=0, stream=None) -> int:
    """chessfad_hvp with host-resident x, v, out (tensors in host memory, or
    addresses) and caller-owned device staging buffers; copies and sweeps of
    consecutive slices overlap."""
    p = ctypes.byref(params) if params is not None else None
    return load().chessfad_hvp_host(fn, n, batch, csize, _addr(x_host), _addr(v_host), _addr(out_host),
                                    _addr(x_dev), _addr(v_dev), _addr(out_dev), p, prec, slices, _stream(stream))


def chessfad_hessian(fn, n, batch, csize, x, H, params=None, prec=FP64, stream=None) -> int:
    p = ctypes.byref(params) if params is not None else None
    return load().chessfad_hessian(fn, n, batch, csize, _addr(x), _addr(H), p, prec, _stream(stream))


def chessfad_hvp_config(fn, n, batch, cfg, x, v, out, params=None, prec=FP64, stream=None) -> int:
    p = ctypes.byref(params) if params is not None else None
    c = ctypes.byref(cfg) if cfg is not None else None
    return load().chessfad_hvp_config(fn, n, batch, c, _addr(x), _addr(v), _addr(out), p, prec, _stream(stream))


def chessfad_hessian_config(fn, n, batch, cfg, x, H, params=None, prec=FP64, stream=None) -> int:
    p = ctypes.byref(params) if params is not None else None
    c = ctypes.byref(cfg) if cfg is not None else None
    return load().chessfad_hessian_config(fn, n, batch, c, _addr(x), _addr(H), p, prec, _stream(stream))


def chessfad_default_config(fn, n, batch, prec) -> Config:
    cfg = Config()
    _check(load().chessfad_default_config(fn, n, batch, prec, ctypes.byref(cfg)), "chessfad_default_config")
    return cfg


def chessfad_resolve_config(fn, n, batch, prec, cfg: Config | None = None, hvp: bool = True) -> Config:
    out = Config()
    _check(load().chessfad_resolve_config(fn, n, batch, prec, 1 if hvp else 0,
                                          ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(out)),
           "chessfad_resolve_config")
    return out


def chessfad_autotune_hessian(fn, n, batch, x, H, params=None, prec=FP64, stream=None) -> Config:
    cfg = Config()
    p = ctypes.byref(params) if params is not None else None
    _check(load().chessfad_autotune_hessian(fn, n, batch, _addr(x), _addr(H), p, prec, _stream(stream),
                                            ctypes.byref(cfg)), "chessfad_autotune_hessian")
    return cfg


def chessfad_autotune_hvp(fn, n, batch, x, v, out, params=None, prec=FP64, stream=None) -> Config:
    cfg = Config()
    p = ctypes.byref(params) if params is not None else None
    _check(load().chessfad_autotune_hvp(fn, n, batch, _addr(x), _addr(v), _addr(out), p, prec, _stream(stream),
                                        ctypes.byref(cfg)), "chessfad_autotune_hvp")
    return cfg


def chessfad_peak_flops(prec) -> float:
    f = ctypes.c_double()
    _check(load().chessfad_peak_flops(prec, ctypes.byref(f)), "chessfad_peak_flops")
    return f.value


def chessfad_peak_info(prec) -> tuple[float, float]:
    """(FMA peak flop/s, SM clock in MHz the fastest run saw)."""
    f = ctypes.c_double()
    mhz = ctypes.c_double()
    _check(load().chessfad_peak_info(prec, ctypes.byref(f), ctypes.byref(mhz)), "chessfad_peak_info")
    return f.value, mhz.value


def chessfad_peak_operand_rates(prec) -> tuple[float, float]:
    """(flop/s with register multipliers, flop/s with literal multipliers) of
    the accumulation-chain FMA shape."""
    r = ctypes.c_double()
    lit = ctypes.c_double()
    _check(load().chessfad_peak_operand_rates(prec, ctypes.byref(r), ctypes.byref(lit)),
           "chessfad_peak_operand_rates")
    return r.value, lit.value


def chessfad_eft(a, b, count, s=None, e=None, p=None, q=None, stream=None) -> int:
    """TwoSum (s, e) and TwoProd (p, q) of float device arrays a, b, elementwise;
    returns the status."""
    return load().chessfad_eft(_addr(a), _addr(b), count, _addr(s), _addr(e), _addr(p), _addr(q), _stream(stream))


def chessfad_compensated_rows(a, b, rows, length, lanes, chunk, out, stream=None) -> int:
    """Dot2 of the rows of a and b (Sum2 of a's rows when b is None) in the
    lane order of the compensated-FP32 row reduction; returns the status."""
    return load().chessfad_compensated_rows(_addr(a), _addr(b), rows, length, lanes, chunk, _addr(out),
                                            _stream(stream))


def chessfad_kernel_info(fn, prec, csize, hvp=True) -> dict:
    regs = ctypes.c_int()
    local = ctypes.c_longlong()
    _check(load().chessfad_kernel_info(fn, prec, csize, int(bool(hvp)), ctypes.byref(regs), ctypes.byref(local)),
           "chessfad_kernel_info")
    return {"registers": regs.value, "local_bytes": local.value}


def chessfad_strerror(status) -> str:
    return strerror(status)


def chessfad_version() -> int:
    return load().chessfad_version()


# ------------------------------------------------------------ conveniences
def _dtype(prec):
    import torch

    return torch.float64 if prec == FP64 else torch.float32


def hvp(fn, x, v, csize=0, params=None, prec=None, stream=None, out=None, cfg=None):
    """out = H(x_p) v_p for device tensors x, v of shape [batch, n] (float64
    for FP64, float32 for FP32_COMP; prec defaults from x's dtype)."""
    import torch

    batch, n = _points(x)
    if prec is None:
        prec = FP64 if x.dtype == torch.float64 else FP32_COMP
    _require(x, "x", _dtype(prec), (batch, n))
    _require(v, "v", _dtype(prec), (batch, n))
    if out is not None:
        _require(out, "out", _dtype(prec), (batch, n))
    _require_fp_extent(fn, n, params)
    _require_cuda(x=x, v=v, out=out)
    if out is None:
        out = torch.empty_like(x)
    if cfg is not None:
        _check(chessfad_hvp_config(fn, n, batch, cfg, x, v, out, params, prec, stream), "chessfad_hvp_config")
    else:
        _check(chessfad_hvp(fn, n, batch, csize, x, v, out, params, prec, stream), "chessfad_hvp")
    return out


def hessian(fn, x, csize=0, params=None, prec=None, stream=None, out=None, cfg=None):
    """H[p] = Hessian of f at x_p for a device tensor x of shape [batch, n]
    (dtypes as for hvp); out is [batch, n, n]."""
    import torch

    batch, n = _points(x)
    if prec is None:
        prec = FP64 if x.dtype == torch.float64 else FP32_COMP
    _require(x, "x", _dtype(prec), (batch, n))
    if out is not None:
        _require(out, "out", _dtype(prec), (batch, n, n))
    _require_fp_extent(fn, n, params)
    _require_cuda(x=x, out=out)
    if out is None:
        out = torch.empty((batch, n, n), dtype=x.dtype, device=x.device)
    if cfg is not None:
        _check(chessfad_hessian_config(fn, n, batch, cfg, x, out, params, prec, stream), "chessfad_hessian_config")
    else:
        _check(chessfad_hessian(fn, n, batch, csize, x, out, params, prec, stream), "chessfad_hessian")
    return out


# ------------------------------------------------------------ uneven batches
REQUEST_DTYPE = None


def request_dtype():
    """numpy dtype with the layout of chessfad_request (fn, n, off, eoff)."""
    import numpy as np

    return np.dtype([("fn", np.int32), ("n", np.int32), ("off", np.int64), ("eoff", np.int64)])


def requests(fns, ns, offs, eoffs=None):
    import numpy as np

    r = np.zeros(len(fns), dtype=request_dtype())
    r["fn"] = fns
    r["n"] = ns
    r["off"] = offs
    r["eoff"] = 0 if eoffs is None else eoffs
    return r


def chessfad_ragged_plan_create(reqs, prec=FP32_COMP, csize=0):
    """Plan handle (int) for a numpy array of requests (see request_dtype)."""
    import numpy as np

    reqs = np.ascontiguousarray(reqs, dtype=request_dtype())
    h = ctypes.c_void_p()
    _check(load().chessfad_ragged_plan_create(reqs.ctypes.data if len(reqs) else None, len(reqs), prec, csize,
                                              ctypes.byref(h)), "chessfad_ragged_plan_create")
    return h.value


def chessfad_ragged_plan_destroy(plan) -> int:
    return load().chessfad_ragged_plan_destroy(plan)


def chessfad_ragged_plan_info(plan) -> dict:
    ws = ctypes.c_size_t()
    nt = ctypes.c_longlong()
    sm = ctypes.c_size_t()
    _check(load().chessfad_ragged_plan_info(plan, ctypes.byref(ws), ctypes.byref(nt), ctypes.byref(sm)),
           "chessfad_ragged_plan_info")
    return {"workspace_bytes": ws.value, "ntiles": nt.value, "smem_bytes": sm.value}


def chessfad_ragged_plan_upload(plan, workspace, workspace_bytes, stream=None) -> int:
    return load().chessfad_ragged_plan_upload(plan, _addr(workspace), workspace_bytes, _stream(stream))


def chessfad_hvp_ragged(plan, xpack, vpack, outpack, params, workspace, workspace_bytes, stream=None) -> int:
    p = ctypes.byref(params) if params is not None else None
    return load().chessfad_hvp_ragged(plan, _addr(xpack), _addr(vpack), _addr(outpack), p, _addr(workspace),
                                      workspace_bytes, _stream(stream))


def chessfad_ragged_plan_group_config(plan, fn, n) -> tuple[int, int, int]:
    """(csize, threads_per_row, A/B tile rows) of the plan's (fn, n) group."""
    c, t, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().chessfad_ragged_plan_group_config(plan, fn, n, ctypes.byref(c), ctypes.byref(t), ctypes.byref(m)),
           "chessfad_ragged_plan_group_config")
    return c.value, t.value, m.value


def chessfad_ragged_autotune(reqs, prec, xpack, vpack, outpack, params, workspace, workspace_bytes,
                             stream=None) -> int:
    """Tune (chunk size, lanes per row) per (function, n range) of the
    requests; returns the number of groups stored."""
    g = ctypes.c_longlong()
    p = ctypes.byref(params) if params is not None else None
    _check(load().chessfad_ragged_autotune(reqs.ctypes.data if len(reqs) else None, len(reqs), prec, _addr(xpack),
                                           _addr(vpack), _addr(outpack), p, _addr(workspace), workspace_bytes,
                                           _stream(stream), ctypes.byref(g)), "chessfad_ragged_autotune")
    return g.value


def chessfad_ragged_tuned_config(prec, fn, n):
    """(csize, threads_per_row, A/B tile KiB) tuned for (prec, fn, n's range),
    or None."""
    c, t, a = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    st = load().chessfad_ragged_tuned_config(prec, fn, n, ctypes.byref(c), ctypes.byref(t), ctypes.byref(a))
    return None if st != SUCCESS else (c.value, t.value, a.value)


def chessfad_hvp_ragged_noalloc(plan, xpack, vpack, outpack, params=None, stream=None) -> int:
    """chessfad_hvp_ragged without a caller workspace: the scratch is the
    library's static device array (see include/chessfad.h)."""
    p = ctypes.byref(params) if params is not None else None
    return load().chessfad_hvp_ragged_noalloc(plan, _addr(xpack), _addr(vpack), _addr(outpack), p, _stream(stream))


class RaggedPlan:
    """Owns a plan and its device workspace (a torch uint8 tensor)."""

    def __init__(self, reqs, prec=FP32_COMP, csize=0, device="cuda", stream=None):
        import torch

        self.prec = prec
        self.handle = chessfad_ragged_plan_create(reqs, prec, csize)
        info = chessfad_ragged_plan_info(self.handle)
        self.info = info
        self.workspace = torch.empty(max(256, info["workspace_bytes"]), dtype=torch.uint8, device=device)
        _check(chessfad_ragged_plan_upload(self.handle, self.workspace, self.workspace.numel(), stream),
               "chessfad_ragged_plan_upload")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def run(self, xpack, vpack, outpack, params=None, stream=None):
        """H v of every request: packed x, v, out (the plan's dtype, one shape,
        contiguous) on the workspace's CUDA device."""
        _require(xpack, "xpack", _dtype(self.prec))
        _require(vpack, "vpack", _dtype(self.prec), xpack.shape)
        _require(outpack, "outpack", _dtype(self.prec), xpack.shape)
        _require_cuda(workspace=self.workspace, xpack=xpack, vpack=vpack, outpack=outpack)
        _check(chessfad_hvp_ragged(self.handle, xpack, vpack, outpack, params, self.workspace,
                                   self.workspace.numel(), stream), "chessfad_hvp_ragged")
        return outpack

    def close(self):
        if self.handle:
            chessfad_ragged_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ user-supplied functions
def chessfad_user_fn_create(source: str, name: str, csize: int, prec: int, log_bytes: int = 16384):
    """Compile a user function (see include/chessfad.h).  Returns
    (status, handle or None, NVRTC log)."""
    h = ctypes.c_void_p()
    log = ctypes.create_string_buffer(log_bytes)
    st = load().chessfad_user_fn_create(source.encode(), name.encode(), csize, prec, ctypes.byref(h), log,
                                        log_bytes)
    return st, (h.value if st == SUCCESS else None), log.value.decode(errors="replace")


def chessfad_user_fn_destroy(handle) -> int:
    return load().chessfad_user_fn_destroy(handle)


def chessfad_user_fn_info(handle, hvp=True) -> dict:
    c, p, r, lb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().chessfad_user_fn_info(handle, int(bool(hvp)), ctypes.byref(c), ctypes.byref(p), ctypes.byref(r),
                                        ctypes.byref(lb)), "chessfad_user_fn_info")
    return {"csize": c.value, "prec": p.value, "registers": r.value, "local_bytes": lb.value}


def chessfad_user_hvp(handle, n, batch, x, v, out, params=None, stream=None) -> int:
    return load().chessfad_user_hvp(handle, n, batch, _addr(x), _addr(v), _addr(out), _addr(params),
                                    _stream(stream))


def chessfad_user_hessian(handle, n, batch, x, H, params=None, stream=None) -> int:
    return load().chessfad_user_hessian(handle, n, batch, _addr(x), _addr(H), _addr(params), _stream(stream))


def chessfad_user_hvp_config(handle, n, batch, cfg, x, v, out, params=None, stream=None) -> int:
    c = ctypes.byref(cfg) if cfg is not None else None
    return load().chessfad_user_hvp_config(handle, n, batch, c, _addr(x), _addr(v), _addr(out), _addr(params),
                                           _stream(stream))


def chessfad_user_hessian_config(handle, n, batch, cfg, x, H, params=None, stream=None) -> int:
    c = ctypes.byref(cfg) if cfg is not None else None
    return load().chessfad_user_hessian_config(handle, n, batch, c, _addr(x), _addr(H), _addr(params),
                                               _stream(stream))


class UserFunction:
    """A user-supplied f compiled for one chunk size and precision.  ``source``
    defines ``template <class R, class X> R name(const X &x, int n, const
    double *params)``; params (optional) is a float64 device tensor passed
    through to f."""

    def __init__(self, source: str, name: str, csize: int = 8, prec: int = FP64):
        st, self.handle, self.log = chessfad_user_fn_create(source, name, csize, prec)
        if st != SUCCESS:
            raise ChessfadError(st, f"chessfad_user_fn_create: {self.log.strip()}")
        self.csize, self.prec, self.name = csize, prec, name

    def info(self, hvp=True) -> dict:
        return chessfad_user_fn_info(self.handle, hvp)

    def hvp(self, x, v, params=None, stream=None, out=None, cfg=None):
        import torch

        batch, n = _points(x)
        _require(x, "x", _dtype(self.prec), (batch, n))
        _require(v, "v", _dtype(self.prec), (batch, n))
        if out is not None:
            _require(out, "out", _dtype(self.prec), (batch, n))
        if params is not None:
            _require(params, "params", torch.float64)
        _require_cuda(x=x, v=v, out=out, params=params)
        if out is None:
            out = torch.empty_like(x)
        _check(chessfad_user_hvp_config(self.handle, n, batch, cfg, x, v, out, params, stream), "chessfad_user_hvp")
        return out

    def hessian(self, x, params=None, stream=None, out=None, cfg=None):
        import torch

        batch, n = _points(x)
        _require(x, "x", _dtype(self.prec), (batch, n))
        if out is not None:
            _require(out, "out", _dtype(self.prec), (batch, n, n))
        if params is not None:
            _require(params, "params", torch.float64)
        _require_cuda(x=x, out=out, params=params)
        if out is None:
            out = torch.empty((batch, n, n), dtype=x.dtype, device=x.device)
        _check(chessfad_user_hessian_config(self.handle, n, batch, cfg, x, out, params, stream),
               "chessfad_user_hessian")
        return out

    def close(self):
        if getattr(self, "handle", None):
            chessfad_user_fn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
