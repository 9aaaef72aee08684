"""Coefficients of phi_neg_f32 in sov_device.cuh (run to reproduce them).

Phi(-x) = phi(x) R(x) with R the Mills ratio, R(x) = sqrt(pi/2) erfcx(x/sqrt(2)).
R is fitted on [0, 12] as a degree-10 polynomial in t = 3 / (3 + x) by least
squares on the relative error (maximum 2e-8 in float64; about 1e-7 when the
kernel evaluates it in float32 by Horner's rule).
"""
import numpy as np
from scipy.special import erfcx


def fit(deg: int = 10, c: float = 3.0, points: int = 200001) -> np.ndarray:
    x = np.linspace(0.0, 12.0, points)
    r = np.sqrt(np.pi / 2) * erfcx(x / np.sqrt(2))
    t = c / (c + x)
    v = np.vander(t, deg + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(v / r[:, None], np.ones_like(r), rcond=None)
    return coef


if __name__ == "__main__":
    co = fit()
    x = np.linspace(0.0, 12.0, 100001)
    r = np.sqrt(np.pi / 2) * erfcx(x / np.sqrt(2))
    print("max relative error (float64):", np.max(np.abs(np.polyval(co[::-1], 3.0 / (3.0 + x)) / r - 1)))
    print(", ".join(f"{c:.9e}f" for c in co.astype(np.float32)))
