"""Coefficients of the central region of ndtri_f32 in sov_device.cuh (run to reproduce them).

For p in (0, 1/2], x = 1 - 2p and w = -log(4 p (1 - p)) = -log(1 - x^2) (the
variable M. Giles uses for the inverse error function, "Approximating the erfinv
function", GPU Computing Gems, 2011), Phi^-1(p) = -sqrt(2) x R(w) with
R(w) = erfinv(x) / x, a smooth function of w.  For w < 5 (p > 0.0017) R is
fitted here as a degree-8 polynomial in w - 2.5 by least squares on the relative
error at Chebyshev nodes (maximum about 2.2e-7 when the kernel evaluates it in
float32 by Horner's rule); the kernel holds the coefficients times -sqrt(2), so
that Phi^-1(p) = x * poly(w - 2.5).  The reference values come from SciPy's float64
normal quantile through p = exp(-w) / (2 (1 + x)), which has no cancellation.
"""
import numpy as np
from scipy.special import ndtri

W_SPLIT, CENTRE, DEG = 5.0, 2.5, 8


def R_of_w(w: np.ndarray) -> np.ndarray:
    x = np.sqrt(-np.expm1(-w))
    p = np.exp(-w) / (2.0 * (1.0 + x))
    out = np.empty_like(w)
    tiny = x < 1e-6  # R(0) = sqrt(pi)/2, first-order series below
    out[~tiny] = -ndtri(p[~tiny]) / np.sqrt(2.0) / x[~tiny]
    out[tiny] = np.sqrt(np.pi) / 2 * (1 + np.pi * x[tiny] ** 2 / 12)
    return out


def fit(points: int = 4000) -> np.ndarray:
    w = np.cos(np.pi * (np.arange(points) + 0.5) / points) * 0.5 * W_SPLIT + 0.5 * W_SPLIT
    r = R_of_w(w)
    v = np.vander(w - CENTRE, DEG + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(v / r[:, None], np.ones_like(r), rcond=None)
    return coef


def float32_error(coef: np.ndarray, points: int = 200001) -> float:
    w = np.linspace(0.0, W_SPLIT, points)
    z = (w - CENTRE).astype(np.float32)
    c = coef.astype(np.float32)
    p = c[-1]
    for a in c[-2::-1]:
        p = (p * z + a).astype(np.float32)
    return float(np.max(np.abs(p.astype(np.float64) / R_of_w(w) - 1)))


if __name__ == "__main__":
    co = fit()
    print("max relative error (float32 Horner):", float32_error(co))
    print(", ".join(f"{c:.9e}f" for c in (-np.sqrt(2.0) * co).astype(np.float32)))
