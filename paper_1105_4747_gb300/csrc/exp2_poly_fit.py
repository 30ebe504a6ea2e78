"""Coefficients of the FMA-pipe exp2 polynomial used by the pair sum's split
exponential mode (tau_extract.cu, exp2_poly).

2^f on [-1/2, 1/2] (the reduced argument of a Cody-Waite split y = n + f) is
fitted by a degree-5 polynomial: least squares on 256 Chebyshev nodes (close
to the minimax fit), converted to the monomial basis and rounded to FP32.
Run as a script to print the coefficients as C float literals.
"""
from __future__ import annotations

import numpy as np

DEGREE = 5
NODES = 256


def coefficients() -> np.ndarray:
    """c[0..DEGREE] (FP32) with 2^f ~ sum_k c[k] f^k on [-1/2, 1/2]."""
    k = np.arange(NODES)
    t = np.cos((2 * k + 1) * np.pi / (2 * NODES))          # Chebyshev nodes of [-1, 1]
    f = 0.5 * t
    cheb = np.polynomial.chebyshev.chebfit(t, np.exp2(f), DEGREE)
    mono_t = np.polynomial.chebyshev.cheb2poly(cheb)        # in t = 2 f
    mono_f = mono_t * (2.0 ** np.arange(DEGREE + 1))
    return mono_f.astype(np.float32)


def exp2_poly_reference(y: np.ndarray, c: np.ndarray | None = None) -> np.ndarray:
    """The kernel's arithmetic in FP32 (numpy), for checking the method:
    y clamped to >= -126, n = round-to-nearest(y), f = y - n, Horner, times 2^n."""
    c = coefficients() if c is None else c
    y = np.maximum(np.asarray(y, dtype=np.float32), np.float32(-126.0))
    n = np.rint(y).astype(np.float32)
    f = (y - n).astype(np.float32)
    p = np.full_like(f, c[DEGREE])
    for k in range(DEGREE - 1, -1, -1):
        p = (p.astype(np.float64) * f.astype(np.float64) + np.float64(c[k])).astype(np.float32)   # fma
    return (p * np.ldexp(np.float32(1.0), n.astype(np.int32))).astype(np.float32)


if __name__ == "__main__":
    for k, v in enumerate(coefficients()):
        h = float(v).hex()
        mant, exp = h.split("p")
        print(f"c{k} = {mant.rstrip('0').rstrip('.')}p{exp}f  ({float(v)!r})")
