"""Writes exp2_table.h: 2^(-k/1024), k = 0 .. 1023, as double-float pairs.

The precise passes of the mean-flux root-find (mean_flux_device.cuh,
exp2_neg_precise) reduce e = 2^-y to 2^-n * 2^(-k/1024) * 2^-g with
|g| <= 2^-11 and read the middle factor from this table.  Each entry is the
value to 50 digits (mpmath) split into hi = nearest float and lo = nearest
float to the remainder, so hi + lo holds it to ~2^-48 relative.  Run as a
script from this directory to regenerate the header.
"""
from __future__ import annotations

import os

import mpmath
import numpy as np

ENTRIES = 1024


def table() -> np.ndarray:
    """[ENTRIES][2] float32: (hi, lo) with hi + lo = 2^(-k/ENTRIES) to ~2^-48."""
    mpmath.mp.dps = 50
    out = np.empty((ENTRIES, 2), dtype=np.float32)
    for k in range(ENTRIES):
        v = mpmath.power(2, mpmath.mpf(-k) / ENTRIES)
        hi = np.float32(float(v))
        lo = np.float32(float(v - mpmath.mpf(float(hi))))
        out[k] = (hi, lo)
    return out


def header(t: np.ndarray) -> str:
    lines = ["// exp2_table.h -- generated by exp2_table_gen.py; do not edit.",
             f"// 2^(-k/{ENTRIES}) for k = 0 .. {ENTRIES - 1} as (hi, lo) floats, hi + lo exact to ~2^-48.",
             "#pragma once", "", f"constexpr int kExp2TabSize = {ENTRIES};", "",
             f"static __device__ const float2 kExp2Tab[{ENTRIES}] = {{"]
    for k in range(ENTRIES):
        lines.append(f"    {{{float(t[k, 0]).hex()}f, {float(t[k, 1]).hex()}f}},".replace("0x", "0x"))
    lines.append("};")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "exp2_table.h"), "w") as f:
        f.write(header(table()))
