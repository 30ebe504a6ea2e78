"""Pins for the FP64 oracle: each checks it against something other than itself.

The oracle (``oracle/lya_oracle.c``) restates Eq. 4-6 and the mean-flux
normalisation of Sec. 2.3.  The checks below come from what the paper and the
mathematics fix: textbook physics (Gunn-Peterson optical depth, photo-
ionisation equilibrium, the hydrogen Doppler width, the critical density),
closed forms obtained by Poisson summation (Jacobi theta functions from
mpmath), invariants (periodic shift, reflection, velocity offsets, Delta^2
scaling), values printed in the paper (tests/golden/paper_values.json) and a
brute-force sum over all periodic images in 30-digit arithmetic.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

import oracle  # noqa: E402
import lya_synth  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
C_CMS = 2.99792458e10
MPC_CM = 3.0856775814913673e24


def _p(**kw):
    base = dict(box=20.0, z=2.5, t_mode=0)
    base.update(kw)
    return oracle.Params(**base)


def _hubble_s(p):
    return oracle.hubble(p) * 1e5 / MPC_CM


def _theta3(z, q):
    return float(mpmath.jtheta(3, z, q))


# --------------------------------------------------------------------------
# units and constants
# --------------------------------------------------------------------------
def test_doppler_width_textbook():
    """b = sqrt(2 k T / m_H) is 12.85 km/s at 1e4 K and scales as T^1/2."""
    g = GOLD["textbook_doppler_b_1e4K_kms"]
    assert oracle.doppler_b(1e4) == pytest.approx(g["value"], rel=5e-4)
    assert oracle.doppler_b(4e4) / oracle.doppler_b(1e4) == pytest.approx(2.0, rel=1e-14)


def test_critical_density_textbook():
    """nbar_H is built on rho_crit = 3 H0^2 / (8 pi G) = 1.87834e-29 h^2 g/cm^3."""
    g = GOLD["textbook_rho_crit_h2_gcm3"]
    p = _p(z=0.0, h=1.0, omega_b=1.0, y_he=0.0)
    rho_crit = oracle.mean_nh(p) * 1.6735575e-24
    assert rho_crit == pytest.approx(g["value"], rel=g["rel"])
    # nbar_H scales with (1+z)^3, Omega_b h^2 and (1 - Y)
    p1, p2 = _p(z=1.0), _p(z=3.0)
    assert oracle.mean_nh(p2) / oracle.mean_nh(p1) == pytest.approx(8.0, rel=1e-14)
    # the hydrogen (not baryon) density: X = 1 - Y with Y near 0.24
    g = GOLD["textbook_mean_nh0"]
    p0 = _p(z=0.0, h=1.0, omega_b=g["omega_b_h2"])
    assert oracle.mean_nh(p0) == pytest.approx(g["value"], rel=g["rel"])


def test_box_velocity_matches_redshift_interval():
    """N du equals c dz/(1+z), dz the redshift span of the box's comoving length.

    The comoving distance comes from integrating c/H(z) (scipy quad), a route
    independent of the oracle's Hubble-law pixel width.
    """
    from scipy.integrate import quad
    from scipy.optimize import brentq
    # boxes small enough that H(z) is constant across them to ~1e-4 (the
    # symmetric span cancels the first-order change of H)
    for box, z, N in [(20.0, 2.5, 256), (5.0, 2.3, 1536), (50.0, 3.0, 512)]:
        p = _p(box=box, z=z)
        h = p.h

        def H(zz):
            return 100.0 * h * math.sqrt(p.omega_m * (1 + zz) ** 3 + p.omega_l)

        L = box / h  # Mpc comoving
        c_kms = C_CMS / 1e5

        def chi(z1):
            return quad(lambda zz: c_kms / H(zz), z, z1, epsabs=0, epsrel=1e-13)[0] - L

        z1 = brentq(chi, z, z + 5.0, xtol=1e-15)
        # centre the interval on z to second order: use the symmetric span
        z0 = brentq(lambda z0: quad(lambda zz: c_kms / H(zz), z0, z, epsrel=1e-13)[0] - L,
                    z - 2.0, z, xtol=1e-15)
        dz = 0.5 * (z1 - z0)
        V = oracle.pixel_velocity(p, N) * N
        assert V == pytest.approx(c_kms * dz / (1 + z), rel=5e-4)


def test_paper_pixel_and_filter_scales():
    """Sec. 4.2: 1 Gpc / 4096 is ~244 kpc; 2 pi / (6.5 Mpc^-1) is ~966 kpc."""
    assert 1e6 / 4096 == pytest.approx(GOLD["pixel_kpc_1gpc_4096"]["value"], abs=0.5)
    kf = GOLD["kf_scale_kpc"]
    # the paper truncates 966.6 to "~966"
    assert int(2 * math.pi / kf["k_F_per_mpc"] * 1e3) == kf["value"]


def test_temperature_pivot():
    """Eq. 5 with the pivot: T rises as (1+delta)^(gamma-1) up to 10, then stays."""
    piv = GOLD["temperature_pivot"]["value"]
    p = _p(t_mode=1, T0=1.5e4, gamma=1.5, delta_pivot=piv)
    t10 = 1.5e4 * 10 ** 0.5
    assert oracle.temperature(p, 1.0) == pytest.approx(1.5e4, rel=1e-15)
    assert oracle.temperature(p, 9.99) == pytest.approx(1.5e4 * 9.99 ** 0.5, rel=1e-15)
    assert oracle.temperature(p, 9.99) < t10
    assert oracle.temperature(p, 10.0) == pytest.approx(t10, rel=1e-15)
    assert oracle.temperature(p, 10.01) == oracle.temperature(p, 10.0)
    assert oracle.temperature(p, 1e3) == oracle.temperature(p, 10.0)
    # inverted relation (gamma < 1) keeps the pivot too
    pi = _p(t_mode=1, T0=1e4, gamma=0.8)
    assert oracle.temperature(pi, 50.0) == pytest.approx(1e4 * 10 ** -0.2, rel=1e-15)
    # stored mode ignores the pivot and returns the given T
    assert oracle.temperature(_p(t_mode=0), 50.0, 3.3e4) == 3.3e4


def test_nhi_photoionisation_equilibrium():
    """Eq. 4 is photo-ionisation equilibrium with the paper's case-A rate.

    n_HI Gamma = alpha_A(T) n_e n_H with alpha_A = 4.17e-13 (T/1e4)^-0.7
    cm^3/s (Sec. 2.3), n_H = nbar_H (1+delta) and n_e = n_H (1 + Y/(2(1-Y)))
    for fully ionised H and He.  The ratio of the oracle's n_HI to this must be
    the same constant for every T, delta, z, Gamma and Omega_b h^2 (which pins
    every exponent of Eq. 4), and that constant must be close to 1 (the
    paper's 7.24e-6 absorbs slightly different atomic inputs).
    """
    Y = 0.24
    ratios = []
    for T, rho, z, g12, ob in [(1e4, 1.0, 3.0, 1.0, 0.0444), (2.5e4, 0.3, 2.5, 0.7, 0.0444),
                               (6e3, 7.0, 2.0, 1.3, 0.05), (1.7e4, 2.0, 4.0, 1.0, 0.04)]:
        p = _p(z=z, gamma12=g12, omega_b=ob)
        n_h = oracle.mean_nh(p) * rho
        n_e = n_h * (1 + Y / (2 * (1 - Y)))
        alpha = 4.17e-13 * (T / 1e4) ** -0.7
        pie = alpha * n_e * n_h / (g12 * 1e-12)
        ratios.append(oracle.nhi(p, rho, T) / pie)
    ratios = np.array(ratios)
    assert np.ptp(ratios) / ratios.mean() < 1e-12
    assert 0.85 < ratios.mean() < 1.2
    assert oracle.nhi(_p(), 0.0, 1e4) == 0.0


# --------------------------------------------------------------------------
# Eq. 6: closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("T", [2.0e3, 1.5e4, 6.0e4])
def test_uniform_field_theta_closed_form(T):
    """Uniform medium, v = 0: tau is constant, tau = c sigma n_HI / H(z) * theta_3.

    Poisson summation of the sampled Gaussian gives sum_m exp(-(m du/b)^2) =
    (b sqrt(pi)/du) theta_3(0, exp(-(pi b/du)^2)); with dR/du = 1/H(z) the
    prefactor of Eq. 6 collapses to the Gunn-Peterson form.
    """
    N = 64
    p = _p()
    rho = np.ones((1, N), np.float32)
    v = np.zeros((1, N), np.float32)
    t = np.full((1, N), T, np.float32)
    tau = oracle.tau(p, rho, v, t)[0]
    b = oracle.doppler_b(float(np.float32(T)))
    du = oracle.pixel_velocity(p, N)
    th = _theta3(0.0, math.exp(-(math.pi * b / du) ** 2))
    n = oracle.nhi(p, 1.0, float(np.float32(T)))
    expect = C_CMS * 4.48e-18 * n / _hubble_s(p) * th
    assert np.ptp(tau) / tau.mean() < 1e-13
    assert tau.mean() == pytest.approx(expect, rel=1e-13)


def test_uniform_field_gunn_peterson_atomic_constants():
    """The Eq. 6 prefactor reproduces the Gunn-Peterson optical depth.

    tau_GP = (pi e^2 f lambda / (m_e c)) n_HI / H(z), with e, m_e, f and lambda
    of H I Ly-alpha taken independently of the paper's sigma_alpha = 4.48e-18
    (which carries three digits, hence the 2e-3 tolerance).
    """
    a = GOLD["lyman_alpha_atomic"]
    N = 128
    p = _p(box=40.0, z=3.0)
    T = 2.0e4
    tau = oracle.tau(p, np.ones((1, N), np.float32), np.zeros((1, N), np.float32),
                     np.full((1, N), T, np.float32))[0]
    n = oracle.nhi(p, 1.0, T)
    b = oracle.doppler_b(T)
    du = oracle.pixel_velocity(p, N)
    th = _theta3(0.0, math.exp(-(math.pi * b / du) ** 2))
    gp = math.pi * a["e_esu"] ** 2 * a["f_lu"] * a["lambda_cm"] / (a["m_e_g"] * a["c_cms"])
    expect = gp * n / _hubble_s(p) * th
    assert tau.mean() == pytest.approx(expect, rel=2e-3)


@pytest.mark.parametrize("b_over_du,vshift", [(0.45, 3.3), (0.8, -17.25), (2.5, 40.6)])
def test_single_absorber_column_conservation(b_over_du, vshift):
    """One absorbing pixel: sum_i tau_i du = c sigma dR n_HI theta_3(pi r/du, q).

    Poisson summation of a Gaussian sampled at offset r from the pixel grid;
    theta_3 carries the sampling correction, which is large when b < du.
    """
    N = 256
    p = _p()
    du = oracle.pixel_velocity(p, N)
    b = b_over_du * du
    T = (b * 1e5) ** 2 * 1.6735575e-24 / (2 * 1.380649e-16)
    T = float(np.float32(T))
    b = oracle.doppler_b(T)
    j0 = 100
    rho = np.zeros((1, N), np.float32)
    rho[0, j0] = 2.0
    v = np.zeros((1, N), np.float32)
    v[0, j0] = np.float32(vshift * du)
    t = np.full((1, N), T, np.float32)
    tau = oracle.tau(p, rho, v, t)[0]
    u = j0 * du + float(v[0, j0])
    r = u - round(u / du) * du
    q = math.exp(-(math.pi * b / du) ** 2)
    n = oracle.nhi(p, 2.0, T)
    dR = oracle.pixel_proper_cm(p, N)
    expect = C_CMS * 4.48e-18 * dR * n / (du * 1e5) * _theta3(math.pi * r / du, q)
    assert tau.sum() == pytest.approx(expect, rel=1e-13)
    # the line sits where u = v_H + v_pec says (sign of v_pec, Sec. 2.3)
    peak = int(np.argmax(tau))
    assert peak == int(round(u / du)) % N


def test_single_absorber_centroid():
    """For b >= 2 du the sampled line's centroid is u_j/du to ~1e-12 pixels."""
    N = 256
    p = _p()
    du = oracle.pixel_velocity(p, N)
    T = 6.0e4  # b ~ 31 km/s ~ 4 du
    for j0, vs in [(10, 55.3), (200, -123.77), (128, 0.0)]:
        rho = np.zeros((1, N), np.float32)
        rho[0, j0] = 1.0
        v = np.zeros((1, N), np.float32)
        v[0, j0] = np.float32(vs)
        tau = oracle.tau(p, rho, v, np.full((1, N), T, np.float32))[0]
        centre = (j0 * du + float(v[0, j0])) / du
        # circular offsets about the expected centre
        m = (np.arange(N) - centre + N / 2) % N - N / 2
        assert float((m * tau).sum() / tau.sum()) == pytest.approx(0.0, abs=1e-9)


def test_column_density_conservation_random_field():
    """sum_i tau_i du = c sigma dR sum_j n_HI,j theta_j: total absorption is conserved."""
    N = 256
    spec = lya_synth.TINY_20MPC
    rho, v, t = lya_synth.skewers(spec, [3])
    p = _p()
    tau = oracle.tau(p, rho, v, t)[0]
    du = oracle.pixel_velocity(p, N)
    dR = oracle.pixel_proper_cm(p, N)
    total = 0.0
    for j in range(N):
        T = float(t[0, j])
        b = oracle.doppler_b(T)
        u = j * du + float(v[0, j])
        r = u - round(u / du) * du
        q = math.exp(-(math.pi * b / du) ** 2)
        total += oracle.nhi(p, float(rho[0, j]), T) * _theta3(math.pi * r / du, q)
    expect = C_CMS * 4.48e-18 * dR / (du * 1e5) * total
    assert tau.sum() == pytest.approx(expect, rel=1e-12)


# --------------------------------------------------------------------------
# Eq. 6: invariants
# --------------------------------------------------------------------------
def _tiny(ids=(0, 1)):
    return lya_synth.skewers(lya_synth.TINY_20MPC, list(ids))


def test_periodic_shift_invariance():
    rho, v, t = _tiny()
    p = _p()
    tau = oracle.tau(p, rho, v, t)
    for s in (1, 37, 255):
        tau_s = oracle.tau(p, np.roll(rho, s, 1), np.roll(v, s, 1), np.roll(t, s, 1))
        np.testing.assert_allclose(tau_s, np.roll(tau, s, 1), rtol=1e-12, atol=0)


def test_reflection_invariance():
    """i -> -i with v -> -v reflects tau."""
    rho, v, t = _tiny()
    p = _p()
    tau = oracle.tau(p, rho, v, t)
    idx = (-np.arange(rho.shape[1])) % rho.shape[1]
    tau_r = oracle.tau(p, rho[:, idx], -v[:, idx], t[:, idx])
    np.testing.assert_allclose(tau_r, tau[:, idx], rtol=1e-11, atol=0)


def test_uniform_velocity_offset_moves_spectrum():
    """Adding k du to every v_pec moves the whole spectrum k pixels redward."""
    rho, v, t = _tiny([5])
    N = rho.shape[1]
    p = _p()
    du = oracle.pixel_velocity(p, N)
    tau = oracle.tau(p, rho, v, t)
    for k in (3, -11):
        v2 = (v.astype(np.float64) + k * du).astype(np.float32)
        tau2 = oracle.tau(p, rho, v2, t)
        # the FP32 rounding of v2 perturbs positions by ~1e-5 km/s
        np.testing.assert_allclose(tau2, np.roll(tau, k, 1), rtol=2e-5, atol=1e-12 * tau.max())


def test_density_squared_scaling():
    """At fixed stored T, scaling 1+delta by a scales tau by a^2 (Eq. 4)."""
    rho, v, t = _tiny([2])
    p = _p()
    tau = oracle.tau(p, rho, v, t)
    tau2 = oracle.tau(p, rho * np.float32(2.0), v, t)
    np.testing.assert_allclose(tau2, 4.0 * tau, rtol=1e-13)


def test_power_law_mode_equals_stored_temperature():
    """Power-law mode with no pivot equals stored mode fed T = T0 rho^(gamma-1)."""
    rho, v, _ = _tiny([4])
    T0, g = 1.5e4, 1.5
    t = (T0 * rho.astype(np.float64) ** (g - 1)).astype(np.float32)
    # stored T is rounded to FP32, the power law is FP64: compare loosely
    a = oracle.tau(_p(t_mode=0), rho, v, t)
    b = oracle.tau(_p(t_mode=1, T0=T0, gamma=g, delta_pivot=np.inf), rho, v)
    np.testing.assert_allclose(a, b, rtol=2e-6)
    # the pivot changes only skewers that reach 1+delta > 10
    c = oracle.tau(_p(t_mode=1, T0=T0, gamma=g, delta_pivot=10.0), rho, v)
    if rho.max() <= 10:
        np.testing.assert_array_equal(b, c)
    else:
        assert not np.allclose(b, c, rtol=1e-9)


def test_brute_force_all_images_30_digits():
    """Tiny random skewers against a 30-digit sum over every periodic image.

    The brute force sums u_j + m V for all images m (not the nearest image),
    so it checks the oracle's wrap as well as its arithmetic.
    """
    rng = np.random.default_rng(7)
    mpmath.mp.dps = 30
    for N, box in [(8, 20.0), (13, 40.0), (16, 30.0)]:
        p = _p(box=box)
        rho = rng.lognormal(0.0, 1.0, (1, N)).astype(np.float32)
        rho[0, 2] = 0.0
        du = oracle.pixel_velocity(p, N)
        V = N * du
        T = rng.uniform(3e3, 1.2e4, (1, N)).astype(np.float32)
        v = rng.uniform(-0.7 * V, 0.7 * V, (1, N)).astype(np.float32)
        # keep every line narrow against the box so the images beyond the
        # nearest are below 1e-20 of it
        assert max(oracle.doppler_b(float(x)) for x in T[0]) < V / 14
        tau = oracle.tau(p, rho, v, T)[0]
        dR = oracle.pixel_proper_cm(p, N)
        pref = mpmath.mpf(C_CMS) * mpmath.mpf(4.48e-18) * mpmath.mpf(dR) / mpmath.sqrt(mpmath.pi)
        for i in range(N):
            acc = mpmath.mpf(0)
            for j in range(N):
                n = oracle.nhi(p, float(rho[0, j]), float(T[0, j]))
                if n == 0.0:
                    continue
                b = mpmath.sqrt(2 * mpmath.mpf(1.380649e-16) * mpmath.mpf(float(T[0, j]))
                                / mpmath.mpf(1.6735575e-24)) / 10 ** 5
                for m in range(-3, 4):
                    d = mpmath.mpf(i) * du - (mpmath.mpf(j) * du + mpmath.mpf(float(v[0, j]))) + m * V
                    acc += mpmath.mpf(n) / (b * 10 ** 5) * mpmath.exp(-(d / b) ** 2)
            # FP64 rounding of d = v_H(i) - u_j is amplified by 2 (d/b)^2 in
            # exp(-(d/b)^2): pixels that only see far line wings carry
            # relative errors up to ~1e-12 * (d/b)^2 / 100
            expect = float(pref * acc)
            rel = 1e-12 if expect > 1e-20 * float(tau.max()) else 1e-10
            assert tau[i] == pytest.approx(expect, rel=rel, abs=1e-300)


# --------------------------------------------------------------------------
# mean-flux rescaling (Sec. 2.3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("Ft", [0.65, 0.72, 0.8, 0.85])
def test_rescale_constant_tau(Ft):
    tau = np.full(1000, 0.37)
    A, _ = oracle.rescale(tau, Ft)
    assert A == pytest.approx(-math.log(Ft) / 0.37, rel=1e-12)


@pytest.mark.parametrize("Ft", [0.65, 0.8])
def test_rescale_two_valued_tau(Ft):
    """tau in {t, 2t}: x = exp(-A t) solves (x + x^2)/2 = Ft, x = (-1 + sqrt(1 + 8 Ft))/2."""
    t1 = 0.9
    tau = np.array([t1, 2 * t1] * 500)
    A, _ = oracle.rescale(tau, Ft)
    x = (-1 + math.sqrt(1 + 8 * Ft)) / 2
    assert math.exp(-A * t1) == pytest.approx(x, rel=1e-12)


def test_rescale_meets_tolerance_and_jensen_start():
    rho, v, t = _tiny()
    tau = oracle.tau(_p(), rho, v, t)
    A, it = oracle.rescale(tau, 0.8, tol=1e-12)
    F = oracle.flux(tau, A)
    assert abs(F.mean() - 0.8) < 1e-12
    A0 = -math.log(0.8) / tau.mean()
    assert A >= A0          # Jensen: the start lies below the root
    assert it <= 12


def test_rescale_rejects_unreachable_target():
    tau = np.array([0.0] * 90 + [1.0] * 10)
    with pytest.raises(oracle.NoConvergence):
        oracle.rescale(tau, 0.85)      # 90 % of pixels keep F = 1 whatever A is
    A, _ = oracle.rescale(tau, 0.92)   # reachable: 0.9 + 0.1 exp(-A) = 0.92
    assert A == pytest.approx(-math.log(0.2), rel=1e-12)
    with pytest.raises(ValueError):
        oracle.rescale(np.zeros(10), 0.8)
    with pytest.raises(ValueError):
        oracle.rescale(np.ones(10), 1.2)


# --------------------------------------------------------------------------
# flux statistics (Sec. 2.3, Sec. 5.2)
# --------------------------------------------------------------------------
def test_tau_eff_paper_value():
    """<F> = 0.72 is quoted as tau_eff = 0.329 (Sec. 2.3)."""
    m = GOLD["mean_flux_z3"]["value"]
    st = oracle.flux_stats(np.full(100, m))
    assert round(st.tau_eff, 3) == GOLD["tau_eff_z3"]["value"]
    assert st.var_flux == pytest.approx(0.0, abs=1e-30)


def _f32_below(x: Fraction) -> np.float32:
    f = np.float32(float(x))
    while Fraction(float(f)) >= x:
        f = np.nextafter(f, np.float32(-1))
    return f


def _f32_at_or_above(x: Fraction) -> np.float32:
    f = np.float32(float(x))
    while Fraction(float(f)) < x:
        f = np.nextafter(f, np.float32(2))
    return f


def test_pdf_bin_edges_exact():
    """Sec. 5.2: 21 bins of width 0.05; bin k holds (2k-1)/40 <= F < (2k+1)/40."""
    g = GOLD["pdf_bins"]
    assert g["n_bins"] == 21 and g["width"] == 0.05
    assert oracle.pdf_bin(0.0) == 0
    assert oracle.pdf_bin(1.0) == 20
    for k in range(20):
        edge = Fraction(2 * k + 1, 40)
        assert oracle.pdf_bin(float(_f32_below(edge))) == k
        assert oracle.pdf_bin(float(_f32_at_or_above(edge))) == k + 1
    F = np.array([_f32_below(Fraction(1, 40)), _f32_at_or_above(Fraction(1, 40)), 1.0, 0.5],
                 dtype=np.float32)
    st = oracle.flux_stats(F)
    assert st.pdf[0] == 1 and st.pdf[1] == 1 and st.pdf[20] == 1 and st.pdf[10] == 1
    assert st.pdf.sum() == 4


def test_flux_stats_moments():
    rng = np.random.default_rng(3)
    F = rng.uniform(0, 1, 10001).astype(np.float32)
    st = oracle.flux_stats(F)
    F64 = F.astype(np.float64)
    assert st.mean_flux == pytest.approx(math.fsum(F64) / F.size, rel=1e-15)
    assert st.var_flux == pytest.approx(np.var(F64), rel=1e-12)
    assert st.tau_eff == pytest.approx(-math.log(st.mean_flux), rel=1e-15)
