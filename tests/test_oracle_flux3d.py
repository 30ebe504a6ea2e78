"""Pins of the oracle's 3D flux power spectrum and Eq. 7 reconstruction:
Parseval, the exact power of a plane wave sampled by every cell, the exact
aliasing term it implies, the expectation for mutually uncorrelated lines
(which Eq. 7 removes), and the shell bookkeeping."""
import math

import numpy as np
import pytest

from oracle import flux3d as f3


def test_parseval_and_mode_count():
    rng = np.random.default_rng(1)
    n, N, L = 8, 32, 50.0
    cells = np.array([(i, j) for i in range(n) for j in range(n) if (i + j) % 3 == 0])
    F = rng.uniform(0.2, 1.0, size=(len(cells), N))
    P_box, _, _, _ = f3.power_terms(F, cells, n, L)
    k, mult = f3.mode_k(n, N, L)
    M = n * n * N
    d = F / F.mean() - 1.0
    # sum over all modes of |G|^2 = M sum over cells of delta^2
    assert float((mult * P_box).sum()) * M ** 2 / L ** 3 == pytest.approx(M * float((d ** 2).sum()), rel=1e-12)
    _, _, _, cnt = f3.shell_average(P_box, P_box, n, N, L)
    assert float(cnt.sum()) == M - 1                                   # every mode but k = 0


def test_plane_wave_fully_sampled():
    n, N, L, a = 8, 64, 100.0, 0.3
    mx, my, mz = 2, 1, 5
    x = np.arange(n)
    z = np.arange(N)
    cells = np.array([(i, j) for i in range(n) for j in range(n)])
    phase = 2 * np.pi * (mx * cells[:, 0, None] / n + my * cells[:, 1, None] / n + mz * z[None, :] / N)
    F = 0.7 * (1.0 + a * np.cos(phase))
    P_box, P_1d, P_2d, P_true = f3.power_terms(F, cells, n, L)
    # the wave's power V a^2 / 4 at +-k0, nothing elsewhere
    assert P_box[mx, my, mz] == pytest.approx(L ** 3 * a * a / 4, rel=1e-10)
    P = P_box.copy()
    P[mx, my, mz] = 0.0
    assert float(P.max()) < 1e-20 * L ** 3
    # every line carries the same 1D wave: P_1D(k_z0) = L a^2 / 4, and with all
    # n^2 cells filled P_2D,w = L^2 / n^2
    assert P_1d[mz] == pytest.approx(L * a * a / 4, rel=1e-10)
    assert P_2d == pytest.approx(L * L / n ** 2, rel=1e-14)
    assert P_true[0, 0, mz] == pytest.approx(-L ** 3 * a * a / (4 * n ** 2), rel=1e-10)


def test_uncorrelated_lines_reconstruct_to_zero():
    rng = np.random.default_rng(7)
    n, N, L = 16, 64, 200.0
    cells = np.array([(i, j) for i in range(n) for j in range(n)])
    ks_all, pt_all, pb_all = [], [], []
    for rep in range(6):
        F = 0.6 * (1.0 + 0.2 * rng.standard_normal((len(cells), N)))
        ks, pt, pb, cnt = f3.flux_power_3d(F, cells, n, L)
        pt_all.append(pt)
        pb_all.append(pb)
    pt = np.mean(pt_all, axis=0)
    pb = np.mean(pb_all, axis=0)
    good = cnt > 200
    # P_box is the aliased 1D power, flat; Eq. 7 removes it to the sampling noise
    assert np.all(pb[good] > 0)
    assert np.all(np.abs(pt[good]) < 8 * pb[good] / np.sqrt(cnt[good] * len(pt_all)))


def test_shell_positions_inside_shells():
    n, N, L = 8, 32, 80.0
    rng = np.random.default_rng(2)
    cells = np.array([(i, (3 * i) % n) for i in range(n)])
    F = rng.uniform(0.3, 1.0, size=(n, N))
    ks, pt, pb, cnt = f3.flux_power_3d(F, cells, n, L)
    kf = 2 * np.pi / L
    b = np.arange(len(ks))
    ok = cnt > 0
    assert np.all(ks[ok] >= b[ok] * kf) and np.all(ks[ok] < (b[ok] + 1) * kf)
