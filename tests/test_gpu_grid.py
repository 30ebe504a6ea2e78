"""The 1536^3 grid: all 2,359,296 rows x 1,536 px of a periodic 1 h^-1 Gpc box at
z = 2.3 (43.5 GB of rho, v_pec, T) extracted in one launch on a borrowed field,
512 random rows (seed 1004) against the FP64 oracle.

Tolerances as in test_gpu_parity: tau relative <= 1e-4 where A tau > 1e-6,
|dF| <= 1e-5 with each side's own A (the GPU's A, over all rows, is checked
by the property that defines it, in FP64)."""
import numpy as np
import pytest

import lya_synth as ls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lya():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 90e9:
        pytest.skip("needs ~90 GB of free device memory")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4747_gb300 as lya
    return lya


def test_grid_1536_full_size(lya):
    import oracle
    import torch
    oracle.build()
    spec = ls.GRID_1536
    S = ls.GRID_1536_ROWS
    rho, v, t = ls.grid_on_device(spec, S, torch)
    field = lya.Field(rho, v, t, box=spec.box, z=spec.z, borrow=True)
    tau = lya.extract_skewers(field, lya.ExtractParams(t_mode=0))
    A, F = lya.rescale_mean_flux(tau, ls.GRID_1536_FT)
    st = lya.flux_stats(F)
    torch.cuda.synchronize()
    # A by the property that defines it (Sec. 2.3), in FP64 on the device
    total = torch.zeros((), dtype=torch.float64, device="cuda")
    flat = tau.reshape(-1)
    for lo in range(0, flat.numel(), 1 << 27):
        total += torch.exp(-A * flat[lo:lo + (1 << 27)].double()).sum()
    assert float(total) / flat.numel() == pytest.approx(ls.GRID_1536_FT, abs=1e-12)
    mean_F = float(F.sum(dtype=torch.float64)) / F.numel()
    assert mean_F == pytest.approx(ls.GRID_1536_FT, abs=1e-7)          # F itself is FP32
    assert st.mean_flux == pytest.approx(ls.GRID_1536_FT, abs=1e-6)
    n_pick, seed = ls.GRID_1536_ORACLE_SUBSET
    ids = ls.random_subset(S, n_pick, seed)
    r_h, v_h, t_h = ls.grid_rows(spec, ids)
    np.testing.assert_array_equal(r_h, rho[torch.as_tensor(ids, device="cuda")].cpu().numpy())
    p = oracle.Params(box=spec.box, z=spec.z, t_mode=0)
    tau_o = oracle.tau(p, r_h, v_h, t_h)
    idx = torch.as_tensor(ids, device="cuda")
    tau_g = tau[idx].double().cpu().numpy()
    mask = A * tau_o > 1e-6
    rel = np.abs(tau_g - tau_o)[mask] / tau_o[mask]
    assert float(rel.max()) <= 1e-4
    F_o = np.exp(-A * tau_o)
    assert float(np.abs(F[idx].cpu().numpy() - F_o).max()) <= 1e-5
    field.close()
    del rho, v, t, tau, F
    torch.cuda.empty_cache()
