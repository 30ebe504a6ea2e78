"""Coefficients of the FP32 erfc used by the pixel-averaged profile
(tau_extract.cu, erfc_pos).

For x >= 0 the kernel writes erfc(x) = t 2^(P(t) - x^2 log2 e) with
t = 1 / (1 + P_SCALE x): the factor e^(-x^2) carries the fall-off, and
P(t) = log2(erfc(x) e^(x^2) / t) is smooth on t in (0, 1] (it tends to a
constant as x -> infinity, where erfc(x) e^(x^2) ~ 1 / (x sqrt(pi))).  P is
fitted here by least squares on Chebyshev nodes of t over x in [0, X_MAX],
with erfc(x) e^(x^2) from scipy's erfcx (double precision), converted to the
monomial basis and rounded to FP32.  Run as a script to print the coefficients as C float
literals (Horner order, highest degree first).
"""
from __future__ import annotations

import numpy as np

DEGREE = 6
P_SCALE = 0.4
X_MAX = 10.0
NODES = 400


def _target(x: np.ndarray) -> np.ndarray:
    from scipy.special import erfcx
    t = 1.0 / (1.0 + P_SCALE * x)
    return np.log2(erfcx(x) / t)


def coefficients() -> np.ndarray:
    """c[0..DEGREE] (FP32) with P(t) ~ sum_k c[k] t^k."""
    t_min = 1.0 / (1.0 + P_SCALE * X_MAX)
    k = np.arange(NODES)
    t = 0.5 * (1.0 + t_min) + 0.5 * (1.0 - t_min) * np.cos((2 * k + 1) * np.pi / (2 * NODES))
    x = (1.0 / t - 1.0) / P_SCALE
    y = _target(x)
    c = np.polynomial.polynomial.polyfit(t, y, DEGREE)
    return c.astype(np.float32)


def erfc_reference(x: np.ndarray, c: np.ndarray | None = None) -> np.ndarray:
    """The kernel's FP32 arithmetic in numpy, for checking the method: t by a
    correctly rounded reciprocal (the kernel's approximate one errs by ~1 ulp
    more), Horner with fma rounded once, 2^z exactly, z = fma(-x log2e, x, P)."""
    c = coefficients() if c is None else c
    f32, f64 = np.float32, np.float64
    x = np.asarray(x, dtype=f32)
    t = (f64(1.0) / (f32(1.0) + f32(P_SCALE) * x).astype(f64)).astype(f32)
    p = np.full_like(t, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p.astype(f64) * t.astype(f64) + f64(c[k])).astype(f32)
    xl = (x * f32(1.4426950408889634)).astype(f32)
    z = (-xl.astype(f64) * x.astype(f64) + p.astype(f64)).astype(f32)
    return (t.astype(f64) * np.exp2(z.astype(f64))).astype(f32)


if __name__ == "__main__":
    for k, v in reversed(list(enumerate(coefficients()))):
        h = float(v).hex()
        mant, exp = h.split("p")
        print(f"c{k} = {mant.rstrip('0').rstrip('.')}p{exp}f  ({float(v)!r})")
