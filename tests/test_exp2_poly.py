"""The FMA-pipe exp2 of the split exponential mode (Cody-Waite reduction and
a fitted degree-5 polynomial): the coefficients compiled into the kernel are
the fitting script's, and the method meets its error bound against numpy's
FP64 exp2 (the kernel's own use of it is checked against the oracle by the
GPU parity tests)."""
import importlib.util
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1105_4747_gb300", "csrc")


def _fit():
    spec = importlib.util.spec_from_file_location("exp2_poly_fit", os.path.join(CSRC, "exp2_poly_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_uses_the_fitted_coefficients():
    fit = _fit()
    src = open(os.path.join(CSRC, "tau_extract.cu")).read()
    body = src[src.index("float exp2_poly(float y)"):]
    body = body[:body.index("\n}\n")]
    lits = [float.fromhex(h) for h in re.findall(r"(0x[0-9a-f.]+p[-+]?\d+)f", body)]
    # the shifter 1.5 * 2^23, then c5 .. c0 in Horner order
    assert lits[0] == 1.5 * 2.0 ** 23
    np.testing.assert_array_equal(np.array(lits[1:][::-1], dtype=np.float32), fit.coefficients())


def test_reduced_range_error():
    fit = _fit()
    f = np.linspace(-0.5, 0.5, 400001, dtype=np.float32)
    got = fit.exp2_poly_reference(f).astype(np.float64)
    ref = np.exp2(f.astype(np.float64))
    assert float(np.max(np.abs(got / ref - 1.0))) < 3.0e-7


def test_full_range_and_exact_powers():
    fit = _fit()
    y = -np.geomspace(1e-6, 125.9, 200001).astype(np.float32)
    got = fit.exp2_poly_reference(y).astype(np.float64)
    ref = np.exp2(y.astype(np.float64))
    assert float(np.max(np.abs(got / ref - 1.0))) < 3.0e-7
    n = -np.arange(0, 127, dtype=np.float32)           # integers: f = 0, 2^n exactly scaled
    np.testing.assert_allclose(fit.exp2_poly_reference(n), np.exp2(n.astype(np.float64)), rtol=2e-7)
    # below -126 the argument is clamped: a tiny positive value, never a NaN or 0 * inf
    assert np.all(fit.exp2_poly_reference(np.float32([-200.0, -1e30])) > 0)


# ---- the root-find's fast-pass exponential (degree 6) ---------------------------

def _fast_pass_body():
    src = open(os.path.join(CSRC, "mean_flux_device.cuh")).read()
    body = src[src.index("float exp2_neg_fast(float t"):]
    return body[:body.index("\n}\n")]


def _exp2_neg_fast_reference(t, a_hi, a_lo, c):
    """exp2_neg_fast's FP32 arithmetic in numpy (fma rounded once via FP64,
    which is exact for these products and sums of two FP32 values)."""
    f32, f64 = np.float32, np.float64
    t = np.asarray(t, dtype=f32)
    y_raw = (t * f32(a_hi)).astype(f32)
    y_hi = np.minimum(y_raw, f32(100.0))
    inner = (t.astype(f64) * f64(a_hi) - y_hi.astype(f64)).astype(f32)      # fma(t, a_hi, -y_hi)
    y_lo = np.where(y_raw <= 100.0, (t.astype(f64) * f64(a_lo) + inner.astype(f64)).astype(f32), f32(0.0))
    nf = np.rint(y_hi).astype(f32)
    f = ((nf - y_hi).astype(f32) - y_lo).astype(f32)
    p = np.full_like(f, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p.astype(f64) * f.astype(f64) + f64(c[k])).astype(f32)
    return (p * np.ldexp(f32(1.0), -nf.astype(np.int32))).astype(f32)


def test_fast_pass_uses_the_fitted_degree6_coefficients():
    fit = _fit()
    lits = [float.fromhex(h) for h in re.findall(r"(0x[0-9a-f.]+p[-+]?\d+)f", _fast_pass_body())]
    # c6 .. c0 in Horner order
    np.testing.assert_array_equal(np.array(lits[::-1], dtype=np.float32), fit.coefficients(6))


def test_fast_pass_error_and_bias():
    """Within 1e-7 of 2^-(t a) (a = A log2 e as a float pair) for t a up to
    60, and unbiased to ~1e-9 on average over a smooth spread of arguments:
    the fast pass's sum of e, and so its A, carry no systematic error above
    that level."""
    fit = _fit()
    c = fit.coefficients(6)
    rng = np.random.default_rng(3)
    A = 4.104274933529672
    a = A * 1.4426950408889634
    a_hi = np.float32(a)
    a_lo = np.float32(a - float(a_hi))
    t = (rng.random(2_000_000) ** 3 * 15.0).astype(np.float32)
    got = _exp2_neg_fast_reference(t, a_hi, a_lo, c).astype(np.float64)
    ref = np.exp(-A * t.astype(np.float64))
    rel = got / ref - 1.0
    assert float(np.abs(rel[t * a < 60]).max()) < 1e-7
    assert abs(float(np.mean(got - ref))) < 3e-9 * float(np.mean(ref))
