"""The precise exponential of the mean-flux root-find (mean_flux_device.cuh,
exp2_neg_precise): its table and its arithmetic, checked on the CPU.

* exp2_table.h is what exp2_table_gen.py writes, and every entry hi + lo holds
  2^(-k/1024) to 2^-47 (50-digit mpmath);
* a float32 restatement of the kernel's steps (numpy; the fused multiply-adds
  as the exact float64 product and sum rounded once to float32) gives
  e_hi + e_lo within 5e-14 of exp(-t a) absolute for every y = t a log2(e)
  below the clamp, and within 5e-14 relative where y <= 4 (e >= 1/16): the
  absolute accuracy of the mean of e that the root-find's certificate assumes
  (kPreciseGErr = 2e-13 covers it and the float-pair sums).  Near e = 1 the
  float pair's last rounding (~2^-46) sets the error; the relative error
  grows as ~1.5e-15 y^2 at large y (the series omits the terms of y_lo, the
  argument's low part, beyond the first) on values that shrink as 2^-y.
"""
import os
import sys

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1105_4747_gb300", "csrc")
sys.path.insert(0, CSRC)
import exp2_table_gen as gen  # noqa: E402

f32 = np.float32


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def exp2_neg_precise(t, a_hi, a_lo, tab):
    """The kernel's steps in float32 (see mean_flux_device.cuh)."""
    t, a_hi, a_lo = f32(t), f32(a_hi), f32(a_lo)
    y_raw = f32(t * a_hi)
    y_hi = min(y_raw, f32(100.0))
    y_lo = fma(t, a_lo, fma(t, a_hi, -y_hi)) if y_raw <= 100.0 else f32(0.0)
    Nf = f32(np.rint(f32(y_hi * f32(1024.0))))
    N = int(Nf)
    r = fma(Nf, f32(-1.0 / 1024.0), y_hi)
    L1, L2 = f32(float.fromhex("0x1.62e430p-1")), f32(float.fromhex("-0x1.05c610p-29"))
    u_hi = f32(-r * L1)
    u_lo = f32(fma(-r, L1, -u_hi) - fma(r, L2, f32(y_lo * L1)))
    d_lo = fma(u_hi, fma(u_hi, fma(u_hi, f32(1.0 / 6.0), f32(0.5)), u_lo), u_lo)
    Tx, Ty = tab[N & 1023]
    P = f32(Tx * u_hi)
    Pe = fma(Tx, u_hi, -P)
    R_hi = f32(Tx + P)
    R_lo = f32(f32(Tx - R_hi) + P)
    R_lo = f32(R_lo + f32(Pe + fma(Tx, d_lo, fma(Ty, u_hi, Ty))))
    scale = f32(2.0 ** -(N >> 10))
    return f32(R_hi * scale), f32(R_lo * scale)


def test_header_is_the_generators_output():
    t = gen.table()
    assert open(os.path.join(CSRC, "exp2_table.h")).read() == gen.header(t)


def test_table_entries_to_2_pow_minus_47():
    mpmath.mp.dps = 40
    t = gen.table()
    for k in range(0, gen.ENTRIES, 7):
        v = mpmath.power(2, mpmath.mpf(-k) / gen.ENTRIES)
        got = mpmath.mpf(float(t[k, 0])) + mpmath.mpf(float(t[k, 1]))
        assert abs(got - v) / v <= 2.0 ** -47


def test_precise_exponential_to_5e14():
    mpmath.mp.dps = 40
    tab = gen.table()
    rng = np.random.default_rng(11)
    log2e = 1.4426950408889634
    worst_rel = worst_abs = 0.0
    for _ in range(3000):
        A = float(10 ** rng.uniform(-2, 1.5))                  # mean-flux constants seen in practice
        t = f32(10 ** rng.uniform(-6, 1.8))                     # optical depths
        a = A * log2e
        a_hi = f32(a)
        a_lo = f32(a - float(a_hi))
        if float(t) * float(a_hi) >= 100.0:
            continue
        eh, el = exp2_neg_precise(t, a_hi, a_lo, tab)
        exact = mpmath.exp(-mpmath.mpf(float(t)) * A)
        err = abs(mpmath.mpf(float(eh)) + mpmath.mpf(float(el)) - exact)
        worst_abs = max(worst_abs, float(err))
        if float(t) * a <= 4.0:
            worst_rel = max(worst_rel, float(err / exact))
    assert worst_abs <= 5e-14, worst_abs
    assert worst_rel <= 5e-14, worst_rel
