"""3D flux power spectrum with the Eq. 7 reconstruction: the CUDA path against
the FP64 oracle (oracle/flux3d.py), shell by shell.

Tolerances: the transforms run in FP32 (relative rounding ~1e-6 of each
mode's amplitude) and the per-plane shell sums in FP32 before FP64 totals, so
P_box agrees to 1e-4 relative; P_true = P_box - (aliasing + noise) cancels
most of P_box for nearly uncorrelated lines, so it is compared to 1e-4 of
P_box.  Mode counts are exact; mean |k| agrees to 1e-5.
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


def flux_lines(lya, n_los, n_pix, box, seed):
    spec = ls.FieldSpec(n_pix=n_pix, box=box, z=2.5, k_j=4.0, sigma_delta=1.5, T0=1.5e4, gamma=1.5, seed=seed)
    rho, v, t = ls.skewers(spec, np.arange(n_los))
    field = lya.Field(rho, v, t, box=box, z=spec.z)
    tau = lya.extract_skewers(field, lya.ExtractParams())
    _, F = lya.rescale_mean_flux(tau, 0.8)
    field.close()
    return F


@pytest.mark.parametrize("n_perp,n_pix,fill,noise,box", [(16, 512, 1.0, 0.0, 200.0), (12, 768, 0.4, 0.05, 200.0),
                                                         (32, 256, 0.3, 0.0, 200.0),
                                                         # the size bench.py times: 4,096 lines of 4,096 px
                                                         # filling a 64 x 64 grid across a 1 h^-1 Gpc box
                                                         (64, 4096, 1.0, 0.0, 1000.0), (64, 4096, 1.0, 0.05, 1000.0)])
def test_flux_power_3d_matches_oracle(lya, n_perp, n_pix, fill, noise, box):
    from oracle import flux3d as f3
    rng = np.random.default_rng(n_perp * 1000 + n_pix)
    all_cells = np.array([(i, j) for i in range(n_perp) for j in range(n_perp)])
    pick = all_cells[rng.permutation(len(all_cells))[: max(2, int(fill * len(all_cells)))]]
    F = flux_lines(lya, len(pick), n_pix, box, seed=40 + n_perp)
    if fill == 1.0 and n_perp == 64:
        # as bench.py calls it: line i at flat cell i (ix * n_perp + iy)
        pick = np.stack([np.arange(len(pick)) // n_perp, np.arange(len(pick)) % n_perp], axis=1)
        k, pt, pb, nm = lya.flux_power_3d(F, np.arange(len(pick)), n_perp, box, noise)
    else:
        k, pt, pb, nm = lya.flux_power_3d(F, pick, n_perp, box, noise)
    ko, pto, pbo, nmo = f3.flux_power_3d(F.cpu().numpy(), pick, n_perp, box, noise)
    assert len(k) == len(ko)
    assert np.array_equal(nm, nmo)
    ok = nmo > 0
    assert np.allclose(k[ok], ko[ok], rtol=1e-5)
    assert np.allclose(pb[ok], pbo[ok], rtol=1e-4)
    assert np.all(np.abs(pt[ok] - pto[ok]) <= 1e-4 * pbo[ok] + 1e-12)


def test_flux_power_3d_errors(lya):
    import torch
    F = torch.ones((4, 100), device="cuda")
    with pytest.raises(lya.LyaError):
        lya.flux_power_3d(F, [0, 1, 2, 3], 8, 100.0)          # 100 = 2^2 5^2
    F = torch.ones((4, 64), device="cuda")
    with pytest.raises(lya.LyaError):
        lya.flux_power_3d(F, [0, 1, 2, 64], 8, 100.0)         # cell outside the 8 x 8 grid
