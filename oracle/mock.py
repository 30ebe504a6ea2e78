"""Mock-spectrum processing and the 1D flux power spectrum (test infrastructure).

Plain FP64 numpy restatement, checked against the CUDA path by the tests;
like the rest of ``oracle`` it is never imported by the product package.

Sec. 4 turns the simulated transmitted flux into spectra that look like a
given instrument's: a Gaussian instrument profile of a given FWHM, resampling
onto the instrument's pixels (given in Angstrom), Gaussian noise of a given
S/N per pixel and, for the large-volume spectra, only the path between the
quasar's rest-frame Ly-alpha and Ly-beta lines less 3000 km/s of proximity
zone.  Sec. 5.3 compares the line-of-sight flux power spectrum.  The paper
gives these steps in words; the definitions below are the readings taken:

  * instrument profile: periodic discrete convolution with the Gaussian
    exp(-(m du)^2 / 2 sigma^2), sigma = FWHM / (2 sqrt(2 ln 2)), over
    |m du| <= nsigma sigma, the weights normalised to sum to one;
  * resampling: input pixel i is the cell [(i - 1/2) du, (i + 1/2) du) of a
    periodic skewer; output pixel k is the cell [(k - 1/2) B, (k + 1/2) B) and
    takes the cell-overlap-weighted mean of the input;
  * path cut: the first floor(min(V, L_cut) / B) output pixels, V = N du;
  * noise: sigma_n = 1 / (S/N) (continuum units) times a standard normal
    deviate, drawn by Box-Muller from Philox4x32-10 (Salmon et al. 2011) with
    key = the 64-bit seed and counter = (output pixel, skewer row, 0, 0); the
    uniforms are u = (top 24 bits of a word + 1/2) 2^-24, exact in FP32;
  * power spectrum: delta_F = F / <F> - 1 with <F> over every pixel given,
    P(k_n) = (du / N) |sum_j delta_j exp(-2 pi i j n / N)|^2 averaged over
    skewers, k_n = 2 pi n / (N du), n = 0 .. N/2 (s/km and km/s).
"""
from __future__ import annotations

import math

import numpy as np

C_KMS = 2.99792458e5
LAMBDA_ALPHA = 1215.67        # Angstrom, Ly-alpha rest wavelength
LAMBDA_BETA = 1025.72         # Angstrom, Ly-beta rest wavelength
PROXIMITY_KMS = 3000.0        # excluded blueward of the quasar's Ly-alpha (Sec. 4)


def fwhm_to_sigma(fwhm: float) -> float:
    return fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def angstrom_to_kms(dlambda: float, z: float) -> float:
    """Velocity width of dlambda Angstrom at the observed Ly-alpha wavelength."""
    return C_KMS * dlambda / (LAMBDA_ALPHA * (1.0 + z))


def lya_lyb_path_kms(proximity: float = PROXIMITY_KMS) -> float:
    """Velocity path between rest-frame Ly-beta and Ly-alpha, less the proximity zone."""
    return C_KMS * math.log(LAMBDA_ALPHA / LAMBDA_BETA) - proximity


# ---- Philox4x32-10 (counter-based generator, Salmon et al. 2011) ---------------------
_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_LO = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Ten Philox rounds on arrays of 32-bit counters; returns four uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint64) & _LO for x in (c0, c1, c2, c3)]
    k0, k1 = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _LO
        hi1, lo1 = p1 >> np.uint64(32), p1 & _LO
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return [x.astype(np.uint32) for x in c]


def normal_deviates(seed: int, rows, n_cols: int) -> np.ndarray:
    """Standard normal deviates [len(rows)][n_cols]: Box-Muller on the first two
    Philox words of counter (column, row low, row high, 0), 24-bit uniforms."""
    rows = np.asarray(rows, dtype=np.int64).ravel()
    kk, rr = np.meshgrid(np.arange(n_cols, dtype=np.uint64), rows.astype(np.uint64), indexing="xy")
    x = philox4x32_10(kk, rr & _LO, rr >> np.uint64(32), np.zeros_like(kk), seed & 0xFFFFFFFF,
                      (seed >> 32) & 0xFFFFFFFF)
    u1 = ((x[0] >> np.uint32(8)).astype(np.float64) + 0.5) * 2.0 ** -24     # in (0, 1)
    u2 = ((x[1] >> np.uint32(8)).astype(np.float64) + 0.5) * 2.0 ** -24
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ---- the processing steps --------------------------------------------------------------
def gaussian_weights(du: float, fwhm: float, nsigma: float = 6.0) -> np.ndarray:
    """Normalised weights w[m], m = -W .. W, of the instrument profile."""
    sig = fwhm_to_sigma(fwhm)
    W = int(math.floor(nsigma * sig / du))
    m = np.arange(-W, W + 1, dtype=np.float64)
    w = np.exp(-0.5 * (m * du / sig) ** 2)
    return w / w.sum()


def convolve(F, du: float, fwhm: float, nsigma: float = 6.0) -> np.ndarray:
    """Periodic convolution of each skewer (rows of F) with the instrument profile."""
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    w = gaussian_weights(du, fwhm, nsigma)
    W = (w.size - 1) // 2
    out = np.zeros_like(F)
    for m in range(-W, W + 1):
        out += w[m + W] * np.roll(F, -m, axis=1)             # out[i] += w[m] F[i + m]
    return out


def resample(F, du: float, B: float, n_out: int) -> np.ndarray:
    """Cell-overlap mean of the periodic input cells over output cells of width B."""
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    N = F.shape[1]
    out = np.empty((F.shape[0], n_out))
    for k in range(n_out):
        a, b = (k - 0.5) * B, (k + 0.5) * B
        i0 = int(math.floor(a / du + 0.5))
        i1 = int(math.ceil(b / du + 0.5)) - 1
        acc = np.zeros(F.shape[0])
        for i in range(i0, i1 + 1):
            lo, hi = max(a, (i - 0.5) * du), min(b, (i + 0.5) * du)
            if hi > lo:
                acc += (hi - lo) * F[:, i % N]
        out[:, k] = acc / B
    return out


def mock_shape(n_pix: int, du: float, bin_kms: float = 0.0, max_kms: float = 0.0) -> int:
    """Output pixels per skewer."""
    B = bin_kms if bin_kms > 0 else du
    L = n_pix * du if max_kms <= 0 else min(n_pix * du, max_kms)
    return int(math.floor(L / B * (1.0 + 1e-12)))


def mock_spectra(F, du: float, fwhm: float = 0.0, bin_kms: float = 0.0, snr: float = 0.0,
                 max_kms: float = 0.0, seed: int = 0, rows=None, nsigma: float = 6.0) -> np.ndarray:
    """Instrument profile -> resampling -> path cut -> noise, per the readings above."""
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    S, N = F.shape
    x = convolve(F, du, fwhm, nsigma) if fwhm > 0 else F
    B = bin_kms if bin_kms > 0 else du
    M = mock_shape(N, du, bin_kms, max_kms)
    y = resample(x, du, B, M)
    if snr > 0:
        r = np.arange(S) if rows is None else rows
        y = y + normal_deviates(seed, r, M) / snr
    return y


def flux_power_1d(F, du: float):
    """(k [s/km], P(k) [km/s]) of the line-of-sight flux contrast, n = 0 .. N/2."""
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    S, N = F.shape
    d = F / F.mean() - 1.0
    X = np.fft.rfft(d, axis=1)
    P = (du / N) * (np.abs(X) ** 2).mean(axis=0)
    k = 2.0 * np.pi * np.arange(P.size) / (N * du)
    return k, P
