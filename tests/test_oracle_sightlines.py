"""Pins of the oracle's Fourier-space sightline generator (Sec. 2.1-2.2):
ensemble statistics of the Gaussian and lognormal fields, the Eq. 3
velocity-density relation and the Eq. 1 smoothing read off the generated
fields, and counter-based reproducibility."""
import math

import numpy as np
import pytest

from oracle import sightlines as sl

BOX, Z, KJ, SIG = 50.0, 2.5, 4.0, 1.5


def test_lognormal_ensemble():
    N, S = 256, 3000
    rho, v = sl.sightlines(np.arange(S), N, BOX, Z, KJ, SIG, seed=21)
    _, _, _, var_b = sl.mode_table(N, BOX, KJ, SIG)
    assert var_b == pytest.approx(SIG ** 2, rel=1e-14)             # no smoothing: sum P_n = sigma^2
    d = np.log(rho) + 0.5 * var_b                                   # the Gaussian field
    per_skewer = (d ** 2).mean(axis=1)                              # E = sum P_n = sigma^2
    assert per_skewer.mean() == pytest.approx(var_b, rel=6 * per_skewer.std() / math.sqrt(S) / var_b)
    assert abs(d.mean()) < 5 * math.sqrt(var_b / S)
    m = rho.mean(axis=1)                                            # <1 + delta> = 1 for the lognormal
    assert m.mean() == pytest.approx(1.0, abs=6 * m.std() / math.sqrt(S))


def test_mode_power_normalisation():
    N, S = 128, 4000
    rho, _ = sl.sightlines(np.arange(S), N, BOX, Z, KJ, SIG, seed=5)
    k, amp, _, var_b = sl.mode_table(N, BOX, KJ, SIG)
    D = np.fft.rfft(np.log(rho) + 0.5 * var_b, axis=1)[:, 1:N // 2]
    est = (np.abs(D) ** 2).mean(axis=0)                             # E|D_n|^2 = (N/2)^2 E|g|^2 P_n = N^2 P_n / 2
    expect = N * N * amp ** 2 / 2.0
    rel = est / expect - 1.0
    assert np.all(np.abs(rel) < 6 / math.sqrt(S))                   # |g|^2 is exponential: sd/mean = 1
    assert np.abs(D[:, 0]).max() > 0 and np.allclose(np.fft.rfft(np.log(rho), axis=1)[:, N // 2].imag, 0, atol=1e-9)


def test_velocity_follows_eq3():
    N = 512
    rho, v = sl.sightlines(np.arange(6), N, BOX, Z, KJ, SIG, seed=9)
    _, _, _, var_b = sl.mode_table(N, BOX, KJ, SIG)
    D = np.fft.rfft(np.log(rho) + 0.5 * var_b, axis=1)[:, 1:N // 2]
    V = np.fft.rfft(v, axis=1)[:, 1:N // 2]
    k = 2 * np.pi * np.arange(1, N // 2) / BOX
    aH = 100.0 * math.sqrt(0.26 * (1 + Z) ** 3 + 0.74) / (1 + Z)
    assert np.allclose(V, 1j * aH * D / k, rtol=1e-9, atol=1e-9 * np.abs(V).max())
    # linear continuity in real space: dv/dx = -aH delta (spectral derivative)
    dvdx = np.fft.irfft(np.fft.rfft(v, axis=1) * 1j * 2 * np.pi * np.arange(N // 2 + 1) / BOX, n=N, axis=1)
    assert np.allclose(dvdx, -aH * (np.log(rho) + 0.5 * var_b), atol=1e-9 * aH)


def test_eq1_smoothing():
    N, kf = 256, 2.0
    r0, v0 = sl.sightlines(np.arange(4), N, BOX, Z, KJ, SIG, seed=3)
    r1, v1 = sl.sightlines(np.arange(4), N, BOX, Z, KJ, SIG, seed=3, k_f=kf)
    _, _, _, var0 = sl.mode_table(N, BOX, KJ, SIG)
    _, _, smooth, var1 = sl.mode_table(N, BOX, KJ, SIG, kf)
    assert var1 < var0
    D0 = np.fft.rfft(np.log(r0) + 0.5 * var0, axis=1)[:, 1:N // 2]
    D1 = np.fft.rfft(np.log(r1) + 0.5 * var1, axis=1)[:, 1:N // 2]
    k = 2 * np.pi * np.arange(1, N // 2) / BOX
    assert np.allclose(D1, D0 / (1 + (k / kf) ** 2), rtol=1e-9, atol=1e-12 * np.abs(D0).max())
    assert np.array_equal(v0, v1)                                   # Eq. 3 uses the unsmoothed density


def test_counter_based_subsets():
    r, v = sl.sightlines(np.arange(10), 64, BOX, Z, KJ, SIG, seed=77)
    r2, v2 = sl.sightlines([3, 7], 64, BOX, Z, KJ, SIG, seed=77)
    assert np.array_equal(r2, r[[3, 7]]) and np.array_equal(v2, v[[3, 7]])
    r3, _ = sl.sightlines([3], 64, BOX, Z, KJ, SIG, seed=78)
    assert not np.array_equal(r3[0], r[3])
