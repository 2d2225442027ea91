"""The error metrics the parity tests and the bench report."""
import numpy as np

from paper_2410_22575_gb300 import metrics


def test_hvp_error_normalisations():
    """Frobenius and spectral normalisations on Hessians with known norms:
    diag(3, 4) has ||H||_F = 5 and ||H||_2 = 4; the spectral-normalised
    error is never below the Frobenius one and at most sqrt(n) above it."""
    H = np.array([[[3.0, 0.0], [0.0, 4.0]]])
    v = np.array([[0.6, 0.8]])
    r_ref = np.einsum("pij,pj->pi", H, v)
    r = r_ref + np.array([[1e-6, 0.0]])
    e = metrics.hvp_errors(r, r_ref, np.array([5.0]), v)
    es = metrics.hvp_errors_spectral(r, r_ref, H, v)
    d = np.linalg.norm(r - r_ref)  # 1e-6 up to the rounding of r_ref + 1e-6
    assert abs(d - 1e-6) < 1e-15
    assert abs(e[0] - d / 5.0) < 1e-20 and abs(es[0] - d / 4.0) < 1e-20
    rng = np.random.Generator(np.random.PCG64(1))
    A = rng.normal(size=(20, 6, 6))
    H = A + A.transpose(0, 2, 1)
    v = rng.normal(size=(20, 6))
    r_ref = np.einsum("pij,pj->pi", H, v)
    r = r_ref + 1e-8 * rng.normal(size=(20, 6))
    e = metrics.hvp_errors(r, r_ref, np.linalg.norm(H, axis=(1, 2)), v)
    es = metrics.hvp_errors_spectral(r, r_ref, H, v)
    assert np.all(es >= e) and np.all(es <= np.sqrt(6) * e * (1 + 1e-12))
