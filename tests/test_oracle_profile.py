"""Pins of the oracle's pixel-averaged line profile (the averaged variant of
Eq. 6: each line's Gaussian averaged over the pixel's velocity cell instead of
sampled at its centre).  Averaging over cells that tile the periodic line
makes the closed forms exact without the theta-function sampling corrections
that the point-sampled profile needs (tests/test_oracle_pins.py)."""
import math

import numpy as np
import pytest

import lya_synth
import oracle

C_CMS = 2.99792458e10
MPC_CM = 3.0856775814913673e24


def _p(**kw):
    base = dict(box=20.0, z=2.5, t_mode=0, profile=1)
    base.update(kw)
    return oracle.Params(**base)


@pytest.mark.parametrize("T", [3.0e3, 1.5e4, 8.0e4])
def test_uniform_field_is_gunn_peterson_exactly(T):
    """Uniform medium, v = 0: tau = c sigma n_HI / H(z) for any b / du."""
    N = 64
    p = _p()
    tau = oracle.tau(p, np.ones((1, N), np.float32), np.zeros((1, N), np.float32),
                     np.full((1, N), T, np.float32))[0]
    n = oracle.nhi(p, 1.0, float(np.float32(T)))
    hz = oracle.hubble(p) * 1e5 / MPC_CM
    expect = C_CMS * 4.48e-18 * n / hz
    assert np.ptp(tau) / tau.mean() < 1e-13
    assert tau.mean() == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("b_over_du,vshift", [(0.2, 3.3), (0.45, -17.25), (2.5, 40.6)])
def test_single_absorber_conserves_column_exactly(b_over_du, vshift):
    N = 256
    p = _p()
    du = oracle.pixel_velocity(p, N)
    b = b_over_du * du
    T = float(np.float32((b * 1e5) ** 2 * 1.6735575e-24 / (2 * 1.380649e-16)))
    j0 = 100
    rho = np.zeros((1, N), np.float32)
    rho[0, j0] = 2.0
    v = np.zeros((1, N), np.float32)
    v[0, j0] = np.float32(vshift * du)
    tau = oracle.tau(p, rho, v, np.full((1, N), T, np.float32))[0]
    n = oracle.nhi(p, 2.0, T)
    dR = oracle.pixel_proper_cm(p, N)
    assert tau.sum() * du * 1e5 == pytest.approx(C_CMS * 4.48e-18 * dR * n, rel=1e-13)
    # the absorption sits in the cell that holds u_j
    u = j0 * du + float(v[0, j0])
    assert int(np.argmax(tau)) == int(math.floor(u / du + 0.5)) % N


def test_random_field_conserves_column_exactly():
    rho, v, t = lya_synth.skewers(lya_synth.TINY_20MPC, [5])
    p = _p()
    N = rho.shape[1]
    tau = oracle.tau(p, rho, v, t)[0]
    du = oracle.pixel_velocity(p, N)
    dR = oracle.pixel_proper_cm(p, N)
    col = sum(oracle.nhi(p, float(r), float(tt)) for r, tt in zip(rho[0], t[0]) if r > 0)
    assert tau.sum() * du * 1e5 == pytest.approx(C_CMS * 4.48e-18 * dR * col, rel=1e-12)


def test_profile_is_the_cell_mean_of_the_sampled_line():
    """For b >> du the cell mean approaches the sampled value: the two
    profiles agree to (du/b)^2 / 12 relative at line centre (Taylor)."""
    N = 256
    du = oracle.pixel_velocity(_p(), N)
    T = 2.0e5                                         # b ~ 57 km/s ~ 7 du
    rho = np.zeros((1, N), np.float32)
    rho[0, 40] = 1.0
    args = (rho, np.zeros((1, N), np.float32), np.full((1, N), T, np.float32))
    t_avg = oracle.tau(_p(), *args)[0]
    t_pt = oracle.tau(_p(profile=0), *args)[0]
    b = oracle.doppler_b(T)
    # at the centre, mean of exp(-(y/b)^2) over |y| < du/2 = 1 - (du/b)^2 / 12 + O((du/b)^4)
    assert t_avg[40] / t_pt[40] == pytest.approx(1.0 - (du / b) ** 2 / 12.0, abs=(du / b) ** 4 / 50)


def test_shift_and_reflection_invariance():
    rho, v, t = lya_synth.skewers(lya_synth.TINY_20MPC, [7])
    p = _p()
    base = oracle.tau(p, rho, v, t)[0]
    s = 37
    shifted = oracle.tau(p, np.roll(rho, s, 1), np.roll(v, s, 1), np.roll(t, s, 1))[0]
    assert np.allclose(shifted, np.roll(base, s), rtol=1e-13, atol=1e-300)
    refl = oracle.tau(p, rho[:, ::-1].copy(), -v[:, ::-1].copy(), t[:, ::-1].copy())[0]
    assert np.allclose(refl, base[::-1], rtol=1e-12, atol=1e-14 * base.max())
