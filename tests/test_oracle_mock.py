"""Pins of the oracle's mock-spectrum processing and 1D flux power spectrum
(Sec. 4, Sec. 5.3), each independent of the oracle's own formulas: paper
values, closed forms, hand-computed small cases, known-answer vectors and
invariants."""
import json
import math
import os

import numpy as np
import pytest

from oracle import mock

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_philox_known_answers():
    for v in GOLD["philox4x32_10_known_answers"]["vectors"]:
        c = [np.array([int(x, 16)], dtype=np.uint64) for x in v["counter"]]
        k = [int(x, 16) for x in v["key"]]
        out = mock.philox4x32_10(*c, *k)
        assert [int(o[0]) for o in out] == [int(x, 16) for x in v["out"]]


def test_normal_deviates_are_standard_and_counter_based():
    g = mock.normal_deviates(12345, np.arange(400), 500)
    n = g.size
    assert abs(g.mean()) < 5 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(np.mean(g ** 4) - 3.0) < 0.05                  # Gaussian kurtosis
    # any subset of rows or columns reproduces the same values
    assert np.array_equal(mock.normal_deviates(12345, [7, 300], 500), g[[7, 300]])
    assert np.array_equal(mock.normal_deviates(12345, [7], 40)[0], g[7, :40])
    assert not np.array_equal(mock.normal_deviates(12346, [7], 40)[0], g[7, :40])


def test_unit_conversions_match_the_paper():
    b = GOLD["instrument_boss_like"]
    assert mock.angstrom_to_kms(b["fwhm_angstrom"], b["z"]) == pytest.approx(b["fwhm_kms"], rel=5e-3)
    assert mock.fwhm_to_sigma(2.0 * math.sqrt(2.0 * math.log(2.0))) == pytest.approx(1.0, rel=1e-15)
    # the Ly-alpha - Ly-beta path: c ln(1215.67 / 1025.72) less the proximity zone
    path = mock.lya_lyb_path_kms(GOLD["proximity_zone_kms"]["value"])
    # dv = c dlambda / lambda from rest-frame Ly-beta to Ly-alpha, integrated numerically
    from scipy.integrate import quad
    full, _ = quad(lambda lam: 2.99792458e5 / lam, 1025.72, 1215.67, epsabs=1e-10)
    assert path == pytest.approx(full - 3000.0, rel=1e-10)
    assert 47000 < path < 48500


def test_convolution_conserves_and_spreads():
    rng = np.random.default_rng(3)
    du, fwhm = 3.0, 20.0
    F = rng.uniform(0.0, 1.0, size=(5, 256))
    c = mock.convolve(F, du, fwhm)
    assert np.allclose(c.sum(axis=1), F.sum(axis=1), rtol=1e-13)          # periodic, normalised
    assert np.allclose(mock.convolve(np.full((2, 64), 0.7), du, fwhm), 0.7, rtol=1e-14)
    spike = np.zeros((1, 512))
    spike[0, 100] = 1.0
    s = mock.convolve(spike, du, fwhm)[0]
    u = (np.arange(512) - 100) * du
    sig = mock.fwhm_to_sigma(fwhm)
    assert s.sum() == pytest.approx(1.0, rel=1e-14)
    assert (s * u).sum() == pytest.approx(0.0, abs=1e-12)                  # centred on the spike
    assert (s * u * u).sum() == pytest.approx(sig * sig, rel=1e-6)         # width sigma (6 sigma window)
    assert s[100] == pytest.approx(du / (math.sqrt(2 * math.pi) * sig), rel=1e-6)


def test_resampling_hand_computed_and_conserving():
    F = np.arange(1.0, 11.0)[None, :]                  # cells [(i - 1/2), (i + 1/2)) of width 1
    out = mock.resample(F, 1.0, 2.5, 4)[0]
    # bin 0 = [-1.25, 1.25): 0.75 of cell -1 (= cell 9, value 10), cell 0, 0.75 of cell 1
    assert out[0] == pytest.approx((0.75 * 10 + 1 + 0.75 * 2) / 2.5, rel=1e-15)
    # bin 1 = [1.25, 3.75): 0.25 of cell 1, cells 2 and 3, 0.25 of cell 4
    assert out[1] == pytest.approx((0.25 * 2 + 3 + 4 + 0.25 * 5) / 2.5, rel=1e-15)
    assert np.array_equal(mock.resample(F, 1.0, 1.0, 10), F)              # same pixels: identity
    rng = np.random.default_rng(4)
    G = rng.uniform(size=(3, 300))
    r = mock.resample(G, 2.0, 7.5, 80)                                      # 80 x 7.5 = 300 x 2
    assert np.allclose(r.sum(axis=1) * 7.5, G.sum(axis=1) * 2.0, rtol=1e-13)


def test_mock_shape_and_noise_level():
    assert mock.mock_shape(4096, 24.0, 73.0) == int(4096 * 24.0 // 73.0)
    assert mock.mock_shape(4096, 24.0, 73.0, max_kms=48000.0) == int(48000.0 // 73.0)
    assert mock.mock_shape(512, 3.0) == 512
    y = mock.mock_spectra(np.full((64, 512), 0.6), 3.0, fwhm=15.0, bin_kms=7.0, snr=5.0, seed=9)
    assert y.shape == (64, mock.mock_shape(512, 3.0, 7.0))
    assert y.mean() == pytest.approx(0.6, abs=5 * 0.2 / math.sqrt(y.size))
    assert y.std() == pytest.approx(0.2, rel=0.03)


def test_flux_power_closed_forms():
    N, du, a, m = 512, 5.0, 0.3, 17
    j = np.arange(N)
    F = 0.7 * (1.0 + a * np.cos(2 * np.pi * m * j / N))[None, :]
    k, P = mock.flux_power_1d(F, du)
    assert k[m] == pytest.approx(2 * np.pi * m / (N * du), rel=1e-15)
    assert P[m] == pytest.approx(N * du * a * a / 4.0, rel=1e-12)
    P2 = P.copy()
    P2[m] = 0.0
    assert np.abs(P2).max() < 1e-20 * P[m] + 1e-25
    rng = np.random.default_rng(5)
    G = rng.uniform(0.1, 1.0, size=(8, 256))
    k, P = mock.flux_power_1d(G, 2.0)
    d = G / G.mean() - 1.0
    V = 256 * 2.0
    parseval = (P[0] + 2 * P[1:-1].sum() + P[-1]) / V            # mean over skewers of mean(delta^2)
    assert parseval == pytest.approx(np.mean(d ** 2), rel=1e-12)
