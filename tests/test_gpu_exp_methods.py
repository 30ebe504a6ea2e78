"""The pair sum's alternative exponentials (Eq. 6): the Gaussian recurrence
and the MUFU / FMA-pipe polynomial split, against the FP64 oracle through the
C ABI, at the same tolerances as the MUFU form: tau relative error <= 1e-4
wherever A tau > 1e-6, |F_gpu - F_oracle| <= 1e-5 with each side solving its
own A."""
import numpy as np
import pytest

import lya_synth as ls
from test_gpu_parity import F_ATOL, assert_tau_close, end_to_end, make_field, oparams

pytestmark = pytest.mark.gpu

METHODS = [1, 2]        # EXP_RECURRENCE, EXP_POLY_SPLIT


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
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("exp_method", METHODS)
@pytest.mark.parametrize("precision", [0, 1])
def test_tiny_box_all_pixels(lya, orc, exp_method, precision):
    spec = ls.TINY_20MPC
    rho, v, t = ls.skewers(spec, np.arange(ls.TINY_20MPC_SKEWERS))
    field = make_field(lya, spec, rho, v, t)
    pg = lya.ExtractParams(precision=precision, exp_method=exp_method)
    tg, A_g, F_g, to, A_o, F_o = end_to_end(lya, orc, field, pg, oparams(orc, spec), rho, v, t,
                                             ls.TINY_20MPC_FT)
    assert_tau_close(tg, to, A_o)
    assert float(np.abs(F_g - F_o).max()) <= F_ATOL


@pytest.mark.parametrize("exp_method", METHODS)
@pytest.mark.parametrize("n_pix,box,T0,gamma", [
    (8192, 50.0, 2.5e4, 1.6),        # b/du ~ 34: every line on the recurrence
    (1024, 50.0, 1.0e4, 1.6),        # a = du sqrt(log2 e)/b on both sides of 0.5
    (512, 1000.0, 1.0e4, 1.0),       # b/du ~ 0.07: every line on the MUFU form
    (16, 20.0, 1.5e4, 1.5),          # shortest skewer (ragged four-pixel tail)
])
def test_geometries(lya, orc, exp_method, n_pix, box, T0, gamma):
    spec = ls.GPC_4096.with_(n_pix=n_pix, box=box, T0=T0, gamma=gamma, seed=11)
    rho, v, _ = ls.skewers(spec, np.arange(3), with_temp=False)
    field = make_field(lya, spec, rho, v, None)
    pg = lya.ExtractParams(t_mode=1, T0=T0, gamma=gamma, exp_method=exp_method)
    tg, A_g, F_g, to, A_o, F_o = end_to_end(lya, orc, field, pg,
                                             oparams(orc, spec, t_mode=1, T0=T0, gamma=gamma),
                                             rho, v, None, 0.7)
    assert_tau_close(tg, to, A_o)
    assert float(np.abs(F_g - F_o).max()) <= F_ATOL


@pytest.mark.parametrize("exp_method", METHODS)
def test_gpc_subset(lya, orc, exp_method):
    """256 random skewers of the 1 h^-1 Gpc, 4,096-pixel field (stored T)."""
    spec = ls.GPC_4096
    ids = ls.random_subset(ls.GPC_4096_SKEWERS, 256, 5)
    rho, v, t = ls.skewers(spec, ids)
    field = make_field(lya, spec, rho, v, t)
    pg = lya.ExtractParams(t_mode=0, exp_method=exp_method)
    tg, A_g, F_g, to, A_o, F_o = end_to_end(lya, orc, field, pg, oparams(orc, spec), rho, v, t,
                                             ls.GPC_4096_FT)
    assert_tau_close(tg, to, A_o)
    assert float(np.abs(F_g - F_o).max()) <= F_ATOL


def test_methods_agree_with_mufu_when_oversampled(lya):
    """Where every line is on the recurrence, the three forms differ only by
    the rounding of their exponentials (a few FP32 ulps of each term)."""
    import torch
    spec = ls.GPC_4096.with_(n_pix=4096, box=100.0, T0=1.5e4, gamma=1.5, seed=12)
    rho, v, _ = ls.skewers(spec, np.arange(64), with_temp=False)
    field = make_field(lya, spec, rho, v, None)
    taus = [lya.extract_skewers(field, lya.ExtractParams(t_mode=1, exp_method=m)) for m in (0, 1, 2)]
    torch.cuda.synchronize()
    ref = taus[0]
    mask = ref > 1e-6
    for tau in taus[1:]:
        rel = ((tau - ref).abs() / ref.clamp_min(1e-30))[mask].max().item()
        assert rel <= 2e-5


def test_rejected_combinations(lya):
    spec = ls.TINY_20MPC
    rho, v, t = ls.skewers(spec, np.arange(4))
    field = make_field(lya, spec, rho, v, t)
    for p in (lya.ExtractParams(precision=2, exp_method=1),
              lya.ExtractParams(profile=lya.PROFILE_AVERAGED, exp_method=2),
              lya.ExtractParams(exp_method=3), lya.ExtractParams(exp_method=-1)):
        with pytest.raises(lya.LyaError):
            lya.extract_skewers(field, p)
    with lya.Server(1 << 30) as srv:
        with pytest.raises(lya.LyaError):
            srv.submit(field, lya.ExtractParams(exp_method=1), np.arange(2), 0.8)
