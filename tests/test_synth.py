"""The seeded input generator: reproducible subsets, the stated statistics and
the linear-theory velocity of Eq. 3 (continuity: dv/dx = -f aH delta)."""
import numpy as np
import pytest

import lya_synth as ls


def test_subsets_reproduce_rows():
    spec = ls.TINY_20MPC
    r_all, v_all, t_all = ls.skewers(spec, np.arange(16))
    ids = [3, 11, 7]
    r, v, t = ls.skewers(spec, ids)
    np.testing.assert_array_equal(r, r_all[ids])
    np.testing.assert_array_equal(v, v_all[ids])
    np.testing.assert_array_equal(t, t_all[ids])
    assert r.dtype == np.float32 and v.dtype == np.float32 and t.dtype == np.float32


def test_ensemble_variance_and_lognormal_mean():
    spec = ls.TINY_20MPC.with_(n_pix=128)
    r, _, _ = ls.skewers(spec, np.arange(2000), with_temp=False)
    delta = np.log(r.astype(np.float64)) + 0.5 * spec.sigma_delta ** 2
    assert delta.var() == pytest.approx(spec.sigma_delta ** 2, rel=0.05)
    assert r.mean() == pytest.approx(1.0, rel=0.05)


def test_velocity_is_linear_theory_convergent_flow():
    """Eq. 3 in 1D: the velocity divergence is -f aH delta (matter falls in)."""
    spec = ls.TINY_20MPC.with_(k_j=2.0)     # smooth field: finite differences work
    r, v, _ = ls.skewers(spec, [0, 1, 2], with_temp=False)
    delta = np.log(r.astype(np.float64)) + 0.5 * spec.sigma_delta ** 2
    dx = spec.box / spec.n_pix
    dvdx = (np.roll(v, -1, 1) - np.roll(v, 1, 1)) / (2 * dx)
    ah = ls.hubble_velocity_per_length(spec)
    c = np.corrcoef(dvdx.ravel(), -ah * delta.ravel())[0, 1]
    assert c > 0.99
    assert np.median(dvdx / (-ah * delta)) == pytest.approx(1.0, rel=0.05)


def test_stored_temperature_power_law():
    spec = ls.TINY_20MPC
    r, _, t = ls.skewers(spec, [1])
    np.testing.assert_allclose(t, spec.T0 * r.astype(np.float64) ** (spec.gamma - 1), rtol=1e-6)


def test_random_subset_sorted_unique():
    s = ls.random_subset(65536, 256, 1001)
    assert s.size == 256 and np.all(np.diff(s) > 0) and s.max() < 65536
