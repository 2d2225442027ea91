"""FP64 CPU oracle for CHESSFAD (arXiv:2410.22575) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg
of ``bench.py`` may import this module.  The product path (the CUDA library and
its binding) never imports, links or runs anything here, and this module
imports nothing from the product package.

The arithmetic lives in ``oracle.c`` (plain C, double precision, no fast-math,
no FMA contraction).  Two independent implementations are exposed:

* O1, closed forms: :func:`value`, :func:`gradient`, :func:`hessian`,
  :func:`hvp`, :func:`hessian_batch`, :func:`hvp_ragged`, :func:`fp_hvp`.  Every chunked
  method of the paper reaches the dense Hessian exactly up to rounding
  (Sec. III-B, Alg. 5), so H(x) and r = H(x) v by their plain definitions are
  the reference.
* O2, the paper's algorithm step by step: the hDual<csize> type of Sec. IV
  (Fig. 1), CHUNK-INIT (Alg. 4), CHUNK-HESS (Alg. 5), SCHUNK-HESS (Alg. 6),
  CHESS-VEC (Alg. 7), SC-HESS-VEC (Alg. 8), with Sec. V operation counters.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (closed-form special values, finite differences,
symmetry, O1 == O2, the four-component rules of Sec. III-A, operation counts
of Sec. V) and ``tests/test_oracle_symbolic.py`` (the closed forms against
symbolic derivatives of each function's formula, evaluated in 40-digit
arithmetic); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

ROSENBROCK, ACKLEY, FLETCHER_POWELL = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, OpenMP when available).

    ``-ffp-contract=off`` keeps a*b+c as two rounded operations on every host
    (gcc contracts to FMA by default on aarch64), so the oracle's rounding is
    the same on x86_64 and Arm.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _FP(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("E", ctypes.c_void_p), ("ld", ctypes.c_int)]


UNARY_OPS = ("sin", "cos", "exp", "sqrt", "log", "tanh", "tan", "recip", "abs")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I = ctypes.c_int
            L = ctypes.c_longlong
            lib.orc_value.restype = ctypes.c_double
            lib.orc_value.argtypes = [I, I, P, P]
            for name in ("orc_gradient", "orc_hessian"):
                getattr(lib, name).argtypes = [I, I, P, P, P]
                getattr(lib, name).restype = I
            lib.orc_hvp_batch.argtypes = [I, I, L, P, P, P, P, P]
            lib.orc_hessian_batch.argtypes = [I, I, L, P, P, P]
            lib.orc_hvp_ragged.argtypes = [L, P, P, P, P, P, P, P, P, P, I, P, P]
            lib.orc_fp_hvp.argtypes = [I, P, P, P, P, P]
            lib.orc_fp_hvp.restype = I
            for name in ("orc_chunk_hess", "orc_schunk_hess"):
                getattr(lib, name).argtypes = [I, I, I, P, P, P]
            for name in ("orc_chess_vec", "orc_sc_hess_vec"):
                getattr(lib, name).argtypes = [I, I, I, P, P, P, P]
            lib.orc_chess_vec_batch.argtypes = [I, I, I, L, P, P, P, P]
            lib.orc_chunk_init.argtypes = [I, P, P, I, I, I]
            lib.orc_chunk_init.restype = None
            for name in ("orc_hd_mul", "orc_hd_add", "orc_hd_div"):
                getattr(lib, name).argtypes = [I, P, P, P]
                getattr(lib, name).restype = None
            for name in UNARY_OPS:
                getattr(lib, f"orc_hd_{name}").argtypes = [I, P, P]
                getattr(lib, f"orc_hd_{name}").restype = None
            lib.orc_hd_pow.argtypes = [I, P, P, ctypes.c_double]
            lib.orc_hd_pow.restype = None
            lib.orc_eval_hd.argtypes = [I, I, I, P, P, P]
            lib.orc_eval_hd.restype = None
            lib.orc_count_reset.restype = None
            lib.orc_count_get.argtypes = [P, P]
            lib.orc_count_get.restype = None
            lib.orc_num_threads.restype = I
            lib.orc_set_num_threads.argtypes = [I]
            lib.orc_set_num_threads.restype = I
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


class FPParams:
    """Fletcher-Powell parameters: A, B (row-major, leading dimension ``ld``,
    leading n x n block used) and E (n entries)."""

    def __init__(self, A, B, E):
        self.A = _f64(A)
        self.B = _f64(B)
        self.E = _f64(E)
        self.ld = self.A.shape[1]

    def _struct(self) -> _FP:
        return _FP(self.A.ctypes.data, self.B.ctypes.data, self.E.ctypes.data, self.ld)


def _params(fn: int, params: FPParams | None):
    if fn == FLETCHER_POWELL:
        if params is None:
            raise ValueError("Fletcher-Powell needs FPParams")
        return ctypes.byref(params._struct())
    return None


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(t: int) -> int:
    """Threads of the OpenMP loops of later calls from this thread; returns
    the previous setting."""
    return _load().orc_set_num_threads(int(t))


# ---------------------------------------------------------------- O1
def value(fn: int, x, params: FPParams | None = None) -> float:
    x = _f64(x)
    return _load().orc_value(fn, x.shape[-1], _ptr(x), _params(fn, params))


def gradient(fn: int, x, params: FPParams | None = None) -> np.ndarray:
    x = _f64(x)
    g = np.empty_like(x)
    if _load().orc_gradient(fn, x.shape[-1], _ptr(x), _params(fn, params), _ptr(g)) != 0:
        raise ValueError("bad function id")
    return g


def hessian(fn: int, x, params: FPParams | None = None) -> np.ndarray:
    x = _f64(x)
    n = x.shape[-1]
    H = np.empty((n, n))
    if _load().orc_hessian(fn, n, _ptr(x), _params(fn, params), _ptr(H)) != 0:
        raise ValueError("bad function id")
    return H


def hvp(fn: int, x, v, params: FPParams | None = None, with_norm: bool = False):
    """Batched r_p = H(x_p) v_p for x, v of shape [batch, n]; optionally also
    ||H(x_p)||_F per point."""
    x = _f64(x)
    v = _f64(v)
    if x.ndim == 1:
        x, v = x[None], v[None]
    batch, n = x.shape
    out = np.empty_like(x)
    hn = np.empty(batch) if with_norm else None
    if _load().orc_hvp_batch(fn, n, batch, _ptr(x), _ptr(v), _params(fn, params), _ptr(out), _ptr(hn)) != 0:
        raise ValueError("oracle failure")
    return (out, hn) if with_norm else out


def hessian_batch(fn: int, x, params: FPParams | None = None) -> np.ndarray:
    x = _f64(x)
    batch, n = x.shape
    H = np.empty((batch, n, n))
    if _load().orc_hessian_batch(fn, n, batch, _ptr(x), _params(fn, params), _ptr(H)) != 0:
        raise ValueError("oracle failure")
    return H


def fp_hvp(x, v, params: FPParams):
    """Fletcher-Powell r = H(x) v and ||H(x)||_F at one point, without forming
    H: (H v)_j = 2 sum_m J_mj (J v)_m + 2 v_j (P^T r)_j, O(n^2) (the norm is
    O(n^3))."""
    x = _f64(x)
    v = _f64(v)
    out = np.empty_like(x)
    hn = ctypes.c_double()
    if _load().orc_fp_hvp(x.shape[-1], _ptr(x), _ptr(v), ctypes.byref(params._struct()), _ptr(out),
                          ctypes.byref(hn)) != 0:
        raise MemoryError
    return out, hn.value


def hvp_ragged(fns, ns, offs, eoffs, xpack, vpack, A=None, B=None, Epack=None, ld=0):
    """Ragged r_q = H_q(x_q) v_q over packed requests; returns (outpack, ||H_q||_F)."""
    fns = np.ascontiguousarray(fns, dtype=np.int32)
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    eoffs = np.ascontiguousarray(eoffs, dtype=np.int64)
    xpack = _f64(xpack)
    vpack = _f64(vpack)
    out = np.zeros_like(xpack)
    hn = np.empty(len(fns))
    A = None if A is None else _f64(A)
    B = None if B is None else _f64(B)
    Epack = None if Epack is None else _f64(Epack)
    rc = _load().orc_hvp_ragged(len(fns), _ptr(fns), _ptr(ns), _ptr(offs), _ptr(eoffs), _ptr(xpack), _ptr(vpack),
                                _ptr(A), _ptr(B), _ptr(Epack), ld, _ptr(out), _ptr(hn))
    if rc != 0:
        raise ValueError("oracle failure")
    return out, hn


# ---------------------------------------------------------------- O2
def chunk_hess(fn: int, x, c: int, params: FPParams | None = None) -> np.ndarray:
    """CHUNK-HESS (Alg. 5) at one point."""
    x = _f64(x)
    n = x.shape[-1]
    H = np.zeros((n, n))
    if _load().orc_chunk_hess(fn, n, c, _ptr(x), _params(fn, params), _ptr(H)) != 0:
        raise MemoryError
    return H


def schunk_hess(fn: int, x, c: int, params: FPParams | None = None) -> np.ndarray:
    """SCHUNK-HESS (Alg. 6) at one point."""
    x = _f64(x)
    n = x.shape[-1]
    H = np.zeros((n, n))
    if _load().orc_schunk_hess(fn, n, c, _ptr(x), _params(fn, params), _ptr(H)) != 0:
        raise MemoryError
    return H


def chess_vec(fn: int, x, v, c: int, params: FPParams | None = None) -> np.ndarray:
    """CHESS-VEC (Alg. 7): one point, or a batch [batch, n] (OpenMP over points)."""
    x = _f64(x)
    v = _f64(v)
    if x.ndim == 2:
        out = np.empty_like(x)
        if _load().orc_chess_vec_batch(fn, x.shape[1], c, x.shape[0], _ptr(x), _ptr(v), _params(fn, params),
                                       _ptr(out)) != 0:
            raise MemoryError
        return out
    out = np.empty_like(x)
    if _load().orc_chess_vec(fn, x.shape[-1], c, _ptr(x), _ptr(v), _params(fn, params), _ptr(out)) != 0:
        raise MemoryError
    return out


def sc_hess_vec(fn: int, x, v, c: int, params: FPParams | None = None) -> np.ndarray:
    """SC-HESS-VEC (Alg. 8) at one point."""
    x = _f64(x)
    v = _f64(v)
    out = np.empty_like(x)
    if _load().orc_sc_hess_vec(fn, x.shape[-1], c, _ptr(x), _ptr(v), _params(fn, params), _ptr(out)) != 0:
        raise MemoryError
    return out


def chunk_init(a, i: int, cstart: int, c: int) -> np.ndarray:
    """CHUNK-INIT (Alg. 4): returns y as an [n, 2c+2] array."""
    a = _f64(a)
    n = a.shape[-1]
    y = np.empty((n, 2 * c + 2))
    _load().orc_chunk_init(n, _ptr(y), _ptr(a), i, cstart, c)
    return y


def eval_hd(fn: int, c: int, y, params: FPParams | None = None) -> np.ndarray:
    """f evaluated on caller-seeded hDuals y ([n, 2c+2])."""
    y = _f64(y)
    out = np.empty(2 * c + 2)
    _load().orc_eval_hd(fn, c, y.shape[0], _ptr(y), _params(fn, params), _ptr(out))
    return out


def hd_op(op: str, c: int, a, b=None) -> np.ndarray:
    """One hDual<c> operation: 'mul', 'add', 'div' (binary, b an hDual),
    'pow' (b the scalar exponent) or one of UNARY_OPS."""
    a = _f64(a)
    r = np.empty(2 * c + 2)
    lib = _load()
    if op in ("mul", "add", "div"):
        b = _f64(b)
        getattr(lib, f"orc_hd_{op}")(c, _ptr(r), _ptr(a), _ptr(b))
    elif op == "pow":
        lib.orc_hd_pow(c, _ptr(r), _ptr(a), float(b))
    else:
        if op not in UNARY_OPS:
            raise ValueError(op)
        getattr(lib, f"orc_hd_{op}")(c, _ptr(r), _ptr(a))
    return r


def count_ops(func, *args, **kw):
    """Run ``func`` (an O2 call, on this thread) and return (result, muls, adds)."""
    lib = _load()
    lib.orc_count_reset()
    res = func(*args, **kw)
    m = ctypes.c_longlong()
    a = ctypes.c_longlong()
    lib.orc_count_get(ctypes.byref(m), ctypes.byref(a))
    return res, m.value, a.value
