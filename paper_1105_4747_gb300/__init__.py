"""GB300-native Lyman-alpha optical depth along skewers.

The data-parallel hot path of the semi-analytic Lyman-alpha forest method of
Greig, Bolton & Wyithe (2011): fluctuating Gunn-Peterson n_HI (Eq. 4-5), the
thermal Doppler profile summed periodically into tau(u_i) (Eq. 6), the
mean-flux rescaling F = exp(-A tau) (Sec. 2.3) and the flux statistics of
Sec. 5.2.  Every step runs in the hand-written sm_103a kernels of
``liblya.so``; this package only marshals arguments through its C ABI
(``include/lya.h``).  PyTorch provides device memory and streams.
"""
from ._binding import (  # noqa: F401
    PREC_F32_COMPENSATED,
    PREC_F32_NAIVE,
    PREC_F64,
    EXP_MUFU,
    EXP_POLY_SPLIT,
    EXP_RECURRENCE,
    PROFILE_AVERAGED,
    PROFILE_SAMPLED,
    ExtractParams,
    Field,
    FluxStats,
    LyaError,
    MockParams,
    Server,
    ServerResult,
    extract_skewers,
    field_pixel_width,
    flux_power_1d,
    flux_power_3d,
    generate_sightlines,
    mock_shape,
    mock_spectra,
    flux_at,
    flux_stats,
    mean_flux_sums,
    mean_flux_start,
    mean_flux_step,
    MeanFluxIter,
    rescale_mean_flux_sharded,
    tau_moments,
    kernel_launches,
    scratch_high_watermark,
    library_path,
    load_library,
    rescale_mean_flux,
    rescale_mean_flux_noalloc,
    rescale_mean_flux_stats,
)
from .distributed import rescale_mean_flux_distributed  # noqa: F401,E402
