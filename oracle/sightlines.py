"""Sightline generation in Fourier space (test infrastructure).

Plain FP64 numpy restatement of the field generation of Sec. 2.1-2.2 for
single lines of sight, checked against the CUDA generator by the tests; the
product package never imports it.

For skewer id s of a field with seed S, N pixels over a periodic box L:
  * modes k_n = 2 pi n / L, n = 1 .. N/2 - 1 (k = 0 and the Nyquist mode are
    zero); the 1D linear power P_n ~ k_n^-1 exp(-(k_n / k_J)^2), scaled so
    that sum_n P_n = sigma_delta^2;
  * amplitudes D_n = (N/2) conj(g_n) sqrt(P_n), g_n = a + i b with a, b
    standard normal from Box-Muller on the first two Philox4x32-10 words of
    counter (n, s low, s high, 0) under key S (uniforms (w >> 8 + 1/2) 2^-24);
  * Eq. 3 in one dimension: V_n = i aH D_n / k_n (f = 1, aH = H(z)/(1+z));
  * Eq. 1 gas smoothing of the density: D_n / (1 + k_n^2 / k_F^2) (k_F = 0:
    none);
  * delta(x_j) and v(x_j) are the inverse real transforms, and
    1 + delta_b = exp(delta_b - sigma_b^2 / 2) with sigma_b^2 the ensemble
    variance sum_n P_n / (1 + k_n^2/k_F^2)^2 (the lognormal stands in for the
    paper's rank-ordered mapping to a hydrodynamical simulation).
"""
from __future__ import annotations

import math

import numpy as np

from .mock import philox4x32_10


def hubble_per_length(z: float, h: float = 0.72, omega_m: float = 0.26, omega_l: float = 0.74) -> float:
    """aH = H(z)/(1+z) in km/s per comoving h^-1 Mpc."""
    return 100.0 * math.sqrt(omega_m * (1.0 + z) ** 3 + omega_l) / (1.0 + z)


def mode_table(n_pix: int, box: float, k_j: float, sigma_delta: float, k_f: float = 0.0):
    """k_n, sqrt(P_n), the Eq. 1 factor and sigma_b^2 for n = 1 .. N/2 - 1."""
    n = np.arange(1, n_pix // 2, dtype=np.float64)
    k = 2.0 * np.pi * n / box
    p = np.exp(-(k / k_j) ** 2) / k
    p *= sigma_delta ** 2 / p.sum()
    smooth = 1.0 / (1.0 + (k / k_f) ** 2) if k_f > 0 else np.ones_like(k)
    return k, np.sqrt(p), smooth, float((p * smooth * smooth).sum())


def gaussian_modes(seed: int, ids, n_modes: int) -> np.ndarray:
    """g_n for n = 1 .. n_modes, one row per skewer id."""
    ids = np.asarray(ids, dtype=np.int64).ravel()
    nn, ss = np.meshgrid(np.arange(1, n_modes + 1, dtype=np.uint64), ids.astype(np.uint64), indexing="xy")
    lo = np.uint64(0xFFFFFFFF)
    w = philox4x32_10(nn, ss & lo, ss >> np.uint64(32), np.zeros_like(nn), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = ((w[0] >> np.uint32(8)).astype(np.float64) + 0.5) * 2.0 ** -24
    u2 = ((w[1] >> np.uint32(8)).astype(np.float64) + 0.5) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2) + 1j * r * np.sin(2.0 * np.pi * u2)


def sightlines(ids, n_pix: int, box: float, z: float, k_j: float, sigma_delta: float, seed: int,
               k_f: float = 0.0, h: float = 0.72, omega_m: float = 0.26, omega_l: float = 0.74):
    """(1 + delta_b, v_pec [km/s]) in FP64, shape [len(ids)][n_pix]."""
    N = n_pix
    k, amp, smooth, var_b = mode_table(N, box, k_j, sigma_delta, k_f)
    g = gaussian_modes(seed, ids, N // 2 - 1)
    D = np.zeros((g.shape[0], N // 2 + 1), dtype=np.complex128)
    D[:, 1:N // 2] = 0.5 * N * np.conj(g) * amp
    V = np.zeros_like(D)
    V[:, 1:N // 2] = 1j * hubble_per_length(z, h, omega_m, omega_l) * D[:, 1:N // 2] / k
    Db = D.copy()
    Db[:, 1:N // 2] *= smooth
    delta_b = np.fft.irfft(Db, n=N, axis=1)
    v = np.fft.irfft(V, n=N, axis=1)
    return np.exp(delta_b - 0.5 * var_b), v
