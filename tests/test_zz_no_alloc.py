"""The allocation-free root-find gives the allocating one's answer.

lya_rescale_mean_flux_noalloc serves callers that cannot allocate device
memory (plug-ins that must not allocate after start-up, services whose memory
budget is spent); its scratch is a fixed device array inside liblya.  Besides
the answers, the test reads the high watermark of the device's default
stream-ordered memory pool through the driver API and that of the
library's own scratch pool (lya_scratch_high_watermark, the pool the
allocating calls draw from): neither grows during a no-alloc call, and the
scratch pool's does during the allocating call on the same input.  This file is named to be
collected last, so a run that stops at the first failure has run every other
test before it.
"""
import math

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


_USED_MEM_HIGH = 8          # CU_MEMPOOL_ATTR_USED_MEM_HIGH (cuda.h)


def _pool_high_watermark():
    """(reset, read) callables for the used-memory high watermark of the
    current device's default memory pool (driver API through ctypes)."""
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0

    def reset():
        zero = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def read():
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value

    return reset, read


def _check_pair(lya, tau, target):
    import torch
    A_ref, F_ref = lya.rescale_mean_flux(tau, target)
    F = torch.empty_like(tau)
    A = lya.rescale_mean_flux_noalloc(tau, target, F)
    torch.cuda.synchronize()
    assert math.isfinite(A)
    assert A == pytest.approx(A_ref, rel=1e-9)
    assert float((F - F_ref).abs().max()) <= 1e-6
    assert float(F.double().mean()) == pytest.approx(target, abs=1e-7)


def test_noalloc_matches_allocating_root_find_twice(lya):
    import torch
    spec = ls.TINY_20MPC
    rho, v, t = ls.skewers(spec, np.arange(ls.TINY_20MPC_SKEWERS))
    field = lya.Field(rho, v, t, box=spec.box, z=spec.z)
    tau = lya.extract_skewers(field, lya.ExtractParams())
    # two calls in a row share the scratch array: the second must not see the first
    _check_pair(lya, tau, ls.TINY_20MPC_FT)
    _check_pair(lya, tau, ls.TINY_20MPC_FT)
    # a larger input (more CTAs than the tiny one) and another target, twice
    g = torch.Generator(device="cuda").manual_seed(3)
    big = torch.rand(3_000_000, device="cuda", generator=g) ** 4 * 5.0
    _check_pair(lya, big, 0.7)
    _check_pair(lya, big, 0.7)


def test_noalloc_draws_nothing_from_the_memory_pool(lya):
    import torch
    g = torch.Generator(device="cuda").manual_seed(5)
    tau = torch.rand(2_000_000, device="cuda", generator=g) ** 3 * 4.0
    F = torch.empty_like(tau)
    torch.cuda.synchronize()
    reset, read = _pool_high_watermark()
    # (a reset watermark starts at the pool's memory in use, normally 0)
    for _ in range(2):
        reset()
        base = read()
        lib_base = lya.scratch_high_watermark(reset=True)
        lib_base = lya.scratch_high_watermark()
        lya.rescale_mean_flux_noalloc(tau, 0.75, F)
        torch.cuda.synchronize()
        assert read() == base
        assert lya.scratch_high_watermark() == lib_base
    # the allocating call on the same input does draw from the library's pool
    # (and not from the default one)
    reset()
    base = read()
    lya.scratch_high_watermark(reset=True)
    lib_base = lya.scratch_high_watermark()
    lya.rescale_mean_flux(tau, 0.75, flux_out=F)
    torch.cuda.synchronize()
    assert lya.scratch_high_watermark() > lib_base
    assert read() == base


def test_noalloc_errors_match(lya):
    import torch
    with pytest.raises(lya.LyaError) as e:
        lya.rescale_mean_flux_noalloc(torch.zeros(100, device="cuda"), 0.8, None)
    assert e.value.status == -1
    tau = torch.tensor([0.0] * 90 + [1.0] * 10, device="cuda")
    with pytest.raises(lya.LyaError) as e:
        lya.rescale_mean_flux_noalloc(tau, 0.85, None)
    assert e.value.status == -4
    with pytest.raises(lya.LyaError):
        lya.rescale_mean_flux_noalloc(tau, 1.5, None)
