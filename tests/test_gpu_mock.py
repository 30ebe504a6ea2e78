"""Mock spectra (Sec. 4) and the 1D flux power spectrum (Sec. 5.3): the CUDA
path against the FP64 oracle (oracle/mock.py), element by element.

Tolerances: processed flux |dF| <= 1e-5 absolute (the method's flux bar; the
profile and resampling sums run in FP32 over at most a few hundred terms);
noise deviates agree to 1e-5 (same Philox words and uniforms; FP32 log and
cos).  Power spectrum: FP32 transforms, so |dP_n| <= 1e-4 P_n + 1e-6 <P>,
where <P> is the mean over n (modes far below the mean carry the FP32
round-off of the transform).
"""
import numpy as np
import pytest

import lya_synth as ls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lya():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4747_gb300 as lya
    return lya


@pytest.fixture(scope="module")
def om():
    from oracle import mock
    return mock


def tiny_flux(lya):
    """F of the 64 x 256 field (stored T), rescaled to <F> = 0.8 on the GPU."""
    spec = ls.TINY_20MPC
    rho, v, t = ls.skewers(spec, np.arange(ls.TINY_20MPC_SKEWERS))
    field = lya.Field(rho, v, t, box=spec.box, z=spec.z)
    tau = lya.extract_skewers(field, lya.ExtractParams())
    _, F = lya.rescale_mean_flux(tau, ls.TINY_20MPC_FT)
    du = lya.field_pixel_width(field)
    field.close()
    return F, du


CASES = [
    dict(fwhm_kms=0.0, bin_kms=0.0),                             # identity
    dict(fwhm_kms=7.0 * 2, bin_kms=0.0),                         # profile only
    dict(fwhm_kms=0.0, bin_kms=19.3),                            # resampling only (non-integer ratio)
    dict(fwhm_kms=30.0, bin_kms=11.0, max_kms=1500.0),           # all three, path cut
    dict(fwhm_kms=60.0, bin_kms=7.7, snr=5.0, seed=77, row0=3),  # with noise
]


@pytest.mark.parametrize("kw", CASES)
def test_mock_spectra_match_oracle(lya, om, kw):
    F, du = tiny_flux(lya)
    p = lya.MockParams(**kw)
    out = lya.mock_spectra(F, du, p).cpu().numpy().astype(np.float64)
    ref = om.mock_spectra(F.cpu().numpy(), du, fwhm=p.fwhm_kms, bin_kms=p.bin_kms, snr=p.snr, max_kms=p.max_kms,
                          seed=p.seed, rows=p.row0 + np.arange(F.shape[0]), nsigma=p.nsigma)
    assert out.shape == ref.shape == (F.shape[0], om.mock_shape(F.shape[1], du, p.bin_kms, p.max_kms))
    assert float(np.abs(out - ref).max()) <= 1e-5


def test_mock_identity_is_exact(lya):
    F, du = tiny_flux(lya)
    out = lya.mock_spectra(F, du, lya.MockParams())
    assert bool((out == F).all())


def test_mock_paper_instruments_on_gpc_skewers(lya, om):
    """The three instruments of Sec. 4 / 5.2 on 64 skewers of the 1 Gpc field at z = 2.5."""
    spec = ls.GPC_4096
    rho, v, t = ls.skewers(spec, np.arange(64))
    field = lya.Field(rho, v, t, box=spec.box, z=spec.z)
    tau = lya.extract_skewers(field, lya.ExtractParams())
    _, F = lya.rescale_mean_flux(tau, ls.GPC_4096_FT)
    du = lya.field_pixel_width(field)
    field.close()
    z = spec.z
    insts = [dict(fwhm_kms=224.0, bin_kms=om.angstrom_to_kms(1.0375, z), snr=5.0, max_kms=om.lya_lyb_path_kms()),
             dict(fwhm_kms=170.0, bin_kms=om.angstrom_to_kms(1.0, z), snr=3.8),
             dict(fwhm_kms=7.0 * 8, bin_kms=om.angstrom_to_kms(0.05, z) * 8, snr=50.0)]
    Fh = F.cpu().numpy()
    for kw in insts:
        p = lya.MockParams(seed=5, **kw)
        out = lya.mock_spectra(F, du, p).cpu().numpy()
        ref = om.mock_spectra(Fh, du, fwhm=p.fwhm_kms, bin_kms=p.bin_kms, snr=p.snr, max_kms=p.max_kms, seed=5)
        assert float(np.abs(out - ref).max()) <= 1e-5


def test_mock_errors(lya):
    import torch
    F = torch.ones((2, 64), device="cuda")
    with pytest.raises(lya.LyaError):
        lya.mock_spectra(F, 1.0, lya.MockParams(fwhm_kms=100.0))        # window wider than the skewer
    with pytest.raises(lya.LyaError):
        lya.mock_spectra(F, 1.0, lya.MockParams(bin_kms=1000.0))        # no output pixel
    with pytest.raises(lya.LyaError):
        lya.mock_spectra(F, -1.0, lya.MockParams())


@pytest.mark.parametrize("n_pix,box", [(256, 20.0), (1536, 1000.0), (4096, 1000.0)])
def test_flux_power_matches_oracle(lya, om, n_pix, box):
    spec = ls.FieldSpec(n_pix=n_pix, box=box, z=2.5, k_j=4.0, sigma_delta=1.5, T0=1.5e4, gamma=1.5, seed=31)
    rho, v, t = ls.skewers(spec, np.arange(33))                         # odd: one skewer rides alone
    field = lya.Field(rho, v, t, box=spec.box, z=spec.z)
    tau = lya.extract_skewers(field, lya.ExtractParams())
    _, F = lya.rescale_mean_flux(tau, 0.8)
    du = lya.field_pixel_width(field)
    field.close()
    k, P, mean = lya.flux_power_1d(F, du)
    kr, Pr = om.flux_power_1d(F.cpu().numpy(), du)
    assert np.allclose(k, kr, rtol=1e-14)
    assert mean == pytest.approx(float(F.double().mean()), rel=1e-9)
    assert np.all(np.abs(P - Pr) <= 1e-4 * Pr + 1e-6 * Pr.mean())


def test_flux_power_closed_form_and_errors(lya):
    import torch
    N, du, a, m = 1024, 3.0, 0.2, 37
    j = torch.arange(N, dtype=torch.float64)
    row = 0.6 * (1.0 + a * torch.cos(2 * np.pi * m * j / N))
    F = row.float().repeat(4, 1).cuda()
    k, P, _ = lya.flux_power_1d(F, du)
    assert P[m] == pytest.approx(N * du * a * a / 4.0, rel=1e-5)
    assert float(np.delete(P, m).max()) < 1e-6 * P[m]
    with pytest.raises(lya.LyaError):
        lya.flux_power_1d(torch.ones((2, 1000), device="cuda"), 1.0)    # 1000 = 2^3 5^3
