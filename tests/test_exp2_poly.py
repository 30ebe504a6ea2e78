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
