"""Error metrics used to compare a computed HVP or Hessian with the oracle.

Per point p (the normalisation the accuracy bounds are stated in):

* HVP:      e_p = ||r_p - r*_p||_2 / (||H*_p||_F ||v_p||_2 + 1e-300)
* Hessian:  e_p = ||H_p - H*_p||_F / (||H*_p||_F + 1e-300)

Frobenius norms bound the spectral norm from above, so these errors are never
smaller than the spectral-normalised ones by more than sqrt(n);
hvp_errors_spectral gives the spectral-normalised HVP error.
"""
from __future__ import annotations

import numpy as np

FP64_BOUND = 1e-12
FP32_COMP_BOUND = 1e-5


def hvp_errors(r, r_ref, hnorm, v) -> np.ndarray:
    r = np.asarray(r, dtype=np.float64)
    r_ref = np.asarray(r_ref, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    num = np.linalg.norm(r - r_ref, axis=-1)
    den = np.asarray(hnorm) * np.linalg.norm(v, axis=-1) + 1e-300
    return num / den


def hvp_errors_spectral(r, r_ref, H_ref, v) -> np.ndarray:
    """e_p = ||r_p - r*_p||_2 / (||H*_p||_2 ||v_p||_2): the spectral-norm
    normalisation (never smaller than the Frobenius one)."""
    r = np.asarray(r, dtype=np.float64)
    r_ref = np.asarray(r_ref, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    num = np.linalg.norm(r - r_ref, axis=-1)
    den = np.linalg.norm(np.asarray(H_ref, dtype=np.float64), ord=2, axis=(-2, -1)) * np.linalg.norm(v, axis=-1)
    return num / (den + 1e-300)


def hessian_errors(H, H_ref) -> np.ndarray:
    H = np.asarray(H, dtype=np.float64)
    H_ref = np.asarray(H_ref, dtype=np.float64)
    num = np.sqrt(((H - H_ref) ** 2).sum(axis=(-1, -2)))
    den = np.sqrt((H_ref ** 2).sum(axis=(-1, -2))) + 1e-300
    return num / den


def ragged_hvp_errors(outpack, refpack, hnorm, vpack, ns, offs) -> np.ndarray:
    outpack = np.asarray(outpack, dtype=np.float64)
    refpack = np.asarray(refpack, dtype=np.float64)
    vpack = np.asarray(vpack, dtype=np.float64)
    d2 = (outpack - refpack) ** 2
    v2 = vpack ** 2
    idx = np.asarray(offs, dtype=np.int64)
    num = np.sqrt(np.add.reduceat(d2, idx)) if len(idx) else np.zeros(0)
    vn = np.sqrt(np.add.reduceat(v2, idx)) if len(idx) else np.zeros(0)
    return num / (np.asarray(hnorm) * vn + 1e-300)


def summary(err: np.ndarray) -> dict:
    err = np.asarray(err)
    if err.size == 0:
        return {"max": 0.0, "median": 0.0}
    return {"max": float(np.max(err)), "median": float(np.median(err))}
