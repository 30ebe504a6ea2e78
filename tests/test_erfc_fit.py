"""The FP32 erfc of the pixel-averaged profile (tau_extract.cu, erfc_pos):
the coefficients compiled into the kernel are the fitting script's, and the
method meets its error bound against scipy's double-precision erfc (the
kernel's own use of it is checked against the FP64 oracle by the GPU parity
tests of the averaged profile)."""
import importlib.util
import os
import re

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1105_4747_gb300", "csrc")


def _fit():
    spec = importlib.util.spec_from_file_location("erfc_fit", os.path.join(CSRC, "erfc_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _kernel_body():
    src = open(os.path.join(CSRC, "tau_extract.cu")).read()
    body = src[src.index("float erfc_pos(float x)"):]
    return body[:body.index("\n}\n")]


def test_kernel_uses_the_fitted_coefficients():
    pytest.importorskip("scipy")
    fit = _fit()
    body = _kernel_body()
    lits = [float.fromhex(h) for h in re.findall(r"(-?0x[0-9a-f.]+p[-+]?\d+)f", body)]
    # c6 .. c0 in Horner order
    np.testing.assert_array_equal(np.array(lits[::-1], dtype=np.float32), fit.coefficients())
    assert "fmaf(0.4f, x, 1.f)" in body and fit.P_SCALE == 0.4


def test_error_bound():
    pytest.importorskip("scipy")
    from scipy.special import erfc
    fit = _fit()
    x = np.linspace(0.0, 9.0, 200001).astype(np.float32)
    got = fit.erfc_reference(x).astype(np.float64)
    ref = erfc(x.astype(np.float64))
    rel = np.abs(got / ref - 1.0)
    assert float(rel[x < 4].max()) < 4e-6
    assert float(rel.max()) < 1e-5
    # the cell differences of the averaged profile: erfc(a) - erfc(a + h) for
    # cells down to a fiftieth of a line width keep their relative accuracy
    a = np.linspace(0.0, 6.0, 2001).astype(np.float32)
    for h in (np.float32(0.02), np.float32(0.5), np.float32(2.0)):
        d = fit.erfc_reference(a).astype(np.float64) - fit.erfc_reference((a + h).astype(np.float32)).astype(np.float64)
        dr = erfc(a.astype(np.float64)) - erfc((a + h).astype(np.float32).astype(np.float64))
        assert float(np.abs(d / dr - 1.0).max()) < (2e-4 if h < 0.1 else 2e-5)


def test_special_values():
    pytest.importorskip("scipy")
    fit = _fit()
    assert float(fit.erfc_reference(np.float32([0.0]))[0]) == pytest.approx(1.0, abs=4e-6)
    # far wing: tiny and positive, monotone
    v = fit.erfc_reference(np.linspace(0, 9, 1001).astype(np.float32)).astype(np.float64)
    assert np.all(np.diff(v) < 0) and np.all(v > 0)
