"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/lya.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lya.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:lya_status|const char\s*\*|uint64_t)\s+(lya_\w+)\s*\(",
                                 text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1105_4747_gb300 import build as b
    b.build()
    import paper_1105_4747_gb300 as lya
    return lya.load_library()


def test_header_declares_the_path():
    names = declared_functions()
    for required in ("lya_create_field", "lya_destroy_field", "lya_extract_skewers",
                     "lya_rescale_mean_flux", "lya_flux_stats", "lya_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in lya.h but not exported"


def test_strerror_and_version(lib):
    assert lib.lya_strerror(0) == b"success"
    assert b"invalid" in lib.lya_strerror(-1)
    assert lib.lya_strerror(-99) == b"unknown status"
    assert b"sm_103a" in lib.lya_version()


def test_host_side_validation_needs_no_device(lib):
    """Invalid arguments return LYA_EINVAL before any CUDA call."""
    import paper_1105_4747_gb300._binding as bnd
    out = ctypes.c_void_p()
    # no descriptor
    assert lib.lya_create_field(None, None, None, None, 0, None, ctypes.byref(out)) == -1
    # odd pixel count / too many pixels / non-positive box
    for kw in (dict(n_pix=255), dict(n_pix=16384), dict(box=0.0), dict(n_skewers=0), dict(z=-1.5)):
        d = dict(box=20.0, z=2.5, h=0.72, omega_m=0.26, omega_l=0.74, omega_b=0.0444, y_he=0.24,
                 n_skewers=4, n_pix=256, has_temp=0)
        d.update(kw)
        desc = bnd._FieldDesc(**d)
        buf = (ctypes.c_float * 4)()
        assert lib.lya_create_field(ctypes.byref(desc), buf, buf, None, 0, None, ctypes.byref(out)) == -1
    A = ctypes.c_double()
    buf = (ctypes.c_float * 4)()
    for target in (0.0, 1.0, 1.5, float("nan")):
        assert lib.lya_rescale_mean_flux(buf, 4, target, 1e-12, 50, ctypes.byref(A), None, None) == -1
    assert lib.lya_rescale_mean_flux(buf, 0, 0.8, 1e-12, 50, ctypes.byref(A), None, None) == -1
    assert lib.lya_rescale_mean_flux(buf, 4, 0.8, 0.0, 50, ctypes.byref(A), None, None) == -1
    st = bnd._FluxStats()
    assert lib.lya_flux_stats(None, 4, ctypes.byref(st), None) == -1
    assert lib.lya_flux_stats(buf, 0, ctypes.byref(st), None) == -1
    p = bnd._ExtractParams(0, 1.5e4, 1.5, 10.0, 1.0, 8.0, 0)
    assert lib.lya_extract_skewers(None, ctypes.byref(p), None, 4, buf, None) == -1


def test_product_does_not_import_the_oracle():
    """The product package never imports, links or reads the oracle."""
    pkg = os.path.join(ROOT, "paper_1105_4747_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "lya_oracle" not in text, f"{f} uses the oracle"


def test_binding_refuses_a_short_or_foreign_flux_out_before_any_launch():
    """The flux pass writes tau.numel() values into flux_out: the binding
    checks its size and device on the host (meta tensors: no GPU, no launch)."""
    import torch
    from paper_1105_4747_gb300 import _binding as b
    tau = torch.empty(100, device="meta")
    with pytest.raises(ValueError, match="100 elements"):
        b._check_out_like(tau, torch.empty(99, device="meta"), "flux_out")
    assert b._check_out_like(tau, torch.empty(100, device="meta"), "flux_out") is not None

    class Elsewhere:                   # a same-size buffer on another device
        device = torch.device("cuda", 1)

        @staticmethod
        def numel():
            return 100
    with pytest.raises(ValueError, match="is on"):
        b._check_out_like(tau, Elsewhere(), "flux_out")
