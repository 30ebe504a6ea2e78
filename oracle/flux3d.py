"""3D flux power spectrum of a set of lines of sight, with the Eq. 7
reconstruction (test infrastructure).

Plain FP64 numpy restatement, checked against the CUDA path by the tests; the
product package never imports it.

The lines of sight run along z through a periodic cube of side L (h^-1 Mpc):
n_los spectra of N pixels, each at a cell (ix, iy) of an n x n transverse
grid (a mock survey).  With delta_F = F / <F> - 1 (<F> over all given pixels):

  * box field: delta_box = delta_F at the lines' cells, 0 elsewhere, on the
    n x n x N grid; G_k its discrete transform, P_box(k) = (V / M^2) |G_k|^2
    with V = L^3 and M = n^2 N cells;
  * weighting field: w = 1 at the lines' cells, 0 elsewhere, on the n x n grid;
    its 2D power (L^2 / n^4) |W(k_perp)|^2 has, over line positions and for
    k_perp != 0, the white level P_2D,w = (L^2 / n^4) sum w^2 = L^2 n_los / n^4,
    which is the factor Eq. 7 needs (the paper calls it the 2D weighting power
    spectrum of the line positions);
  * 1D power of the spectra: P_1D(k_par) = (L / N^2) <|D(k_par)|^2> over the
    lines (D the transform of one line's delta_F);
  * noise: P_N = (L / N) sigma_N^2 P_2D,w(k_perp) for white noise of rms
    sigma_N per pixel in delta_F (0 for noiseless spectra);
  * Eq. 7: P_true(k) = P_box(k) - P_1D(k_par) P_2D,w(k_perp) - P_N(k);
  * spherical average: shells [b k_f, (b + 1) k_f), k_f = 2 pi / L, over the
    modes with k > 0 (the k_par > 0 half-space counted twice, except the
    k_par = 0 and Nyquist planes); each shell reports the mean |k|, the mean
    P_true, the mean P_box and the number of modes.

With these normalisations P_1D P_2D,w is the expectation of P_box, at every
k, for lines whose spectra are uncorrelated with one another: the aliased
line-of-sight power that Eq. 7 removes.
"""
from __future__ import annotations

import math

import numpy as np


def _deltas(F):
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    return F / F.mean() - 1.0


def power_terms(F, cells, n_perp: int, L: float, noise_sigma: float = 0.0):
    """(P_box, P_1D, P_2D_w, P_true) on the half-space grid [n, n, N/2 + 1]."""
    d = _deltas(F)
    S, N = d.shape
    cells = np.asarray(cells, dtype=np.int64).reshape(S, 2)
    grid = np.zeros((n_perp, n_perp, N))
    grid[cells[:, 0], cells[:, 1], :] += d
    G = np.fft.rfftn(grid)                                   # axes (x, y, z): rfft along z
    M = n_perp * n_perp * N
    P_box = (L ** 3 / M ** 2) * np.abs(G) ** 2
    D = np.fft.rfft(d, axis=1)
    P_1d = (L / N ** 2) * (np.abs(D) ** 2).mean(axis=0)      # [N/2 + 1]
    w = np.zeros((n_perp, n_perp))
    np.add.at(w, (cells[:, 0], cells[:, 1]), 1.0)
    P_2d = (L ** 2 / n_perp ** 4) * float((w * w).sum())     # white level of the weights
    P_noise = (L / N) * noise_sigma ** 2 * P_2d
    P_true = P_box - P_1d[None, None, :] * P_2d - P_noise
    return P_box, P_1d, P_2d, P_true


def mode_index2(n_perp: int, N: int):
    """|m|^2 = mx^2 + my^2 + mz^2 (integer mode numbers) over the half-space grid,
    and each mode's multiplicity (k_par = 0 and Nyquist planes once, others twice)."""
    mx = np.fft.fftfreq(n_perp, d=1.0 / n_perp).astype(np.int64)
    mz = np.arange(N // 2 + 1, dtype=np.int64)
    m2 = mx[:, None, None] ** 2 + mx[None, :, None] ** 2 + mz[None, None, :] ** 2
    mult = np.full(N // 2 + 1, 2.0)
    mult[0] = 1.0
    if N % 2 == 0:
        mult[N // 2] = 1.0
    return m2, np.broadcast_to(mult[None, None, :], m2.shape)


def mode_k(n_perp: int, N: int, L: float):
    """|k| (h/Mpc) of every mode of the half-space grid, and its multiplicity."""
    m2, mult = mode_index2(n_perp, N)
    return np.sqrt(m2) * (2.0 * np.pi / L), mult


def shell_average(P_true, P_box, n_perp: int, N: int, L: float):
    """Per shell b (b <= |m| < b + 1 in units of k_f = 2 pi / L): (mean |k|,
    mean P_true, mean P_box, number of modes)."""
    m2, mult = mode_index2(n_perp, N)
    b = np.floor(np.sqrt(m2)).astype(np.int64)                  # integer square root, corrected
    b[(b + 1) ** 2 <= m2] += 1
    b[b ** 2 > m2] -= 1
    k = np.sqrt(m2) * (2.0 * np.pi / L)
    keep = m2 > 0
    nb = int(b[keep].max()) + 1
    cnt = np.bincount(b[keep], weights=mult[keep], minlength=nb)
    ks = np.bincount(b[keep], weights=(mult * k)[keep], minlength=nb)
    pt = np.bincount(b[keep], weights=(mult * P_true)[keep], minlength=nb)
    pb = np.bincount(b[keep], weights=(mult * P_box)[keep], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ks / cnt, pt / cnt, pb / cnt, cnt


def flux_power_3d(F, cells, n_perp: int, L: float, noise_sigma: float = 0.0):
    """The shell-averaged reconstructed 3D flux power spectrum (Eq. 7)."""
    N = np.atleast_2d(F).shape[1]
    P_box, _, _, P_true = power_terms(F, cells, n_perp, L, noise_sigma)
    return shell_average(P_true, P_box, n_perp, N, L)
