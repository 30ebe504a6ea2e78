"""Coefficients of the FMA-pipe exp2 polynomials: degree 5 for the pair
sum's split exponential mode (tau_extract.cu, exp2_poly), degree 6 for the
mean-flux root-find's fast pass (mean_flux_device.cuh, exp2_neg_fast).

2^f on [-1/2, 1/2] (the reduced argument of a Cody-Waite split y = n + f) is
fitted by least squares on 256 Chebyshev nodes (close to the minimax fit),
converted to the monomial basis and rounded to FP32.  Run as a script to
print both sets as C float literals.
"""
from __future__ import annotations

import numpy as np

DEGREE = 5
NODES = 256


def coefficients(degree: int = DEGREE) -> np.ndarray:
    """c[0..degree] (FP32) with 2^f ~ sum_k c[k] f^k on [-1/2, 1/2]."""
    k = np.arange(NODES)
    t = np.cos((2 * k + 1) * np.pi / (2 * NODES))          # Chebyshev nodes of [-1, 1]
    f = 0.5 * t
    cheb = np.polynomial.chebyshev.chebfit(t, np.exp2(f), degree)
    mono_t = np.polynomial.chebyshev.cheb2poly(cheb)        # in t = 2 f
    mono_f = mono_t * (2.0 ** np.arange(degree + 1))
    return mono_f.astype(np.float32)


def exp2_poly_reference(y: np.ndarray, c: np.ndarray | None = None) -> np.ndarray:
    """The kernel's arithmetic in FP32 (numpy), for checking the method:
    y clamped to >= -126, n = round-to-nearest(y), f = y - n, Horner, times 2^n."""
    c = coefficients() if c is None else c
    y = np.maximum(np.asarray(y, dtype=np.float32), np.float32(-126.0))
    n = np.rint(y).astype(np.float32)
    f = (y - n).astype(np.float32)
    d = len(c) - 1
    p = np.full_like(f, c[d])
    for k in range(d - 1, -1, -1):
        p = (p.astype(np.float64) * f.astype(np.float64) + np.float64(c[k])).astype(np.float32)   # fma
    return (p * np.ldexp(np.float32(1.0), n.astype(np.int32))).astype(np.float32)


if __name__ == "__main__":
    for degree in (DEGREE, 6):
        print(f"degree {degree}:")
        for k, v in enumerate(coefficients(degree)):
            h = float(v).hex()
            mant, exp = h.split("p")
            print(f"  c{k} = {mant.rstrip('0').rstrip('.')}p{exp}f  ({float(v)!r})")
