"""ctypes binding of liblya.so: argument marshalling only.

Names mirror the C ABI in ``include/lya.h``.  Device buffers are torch CUDA
tensors; host buffers are numpy arrays (or CPU tensors).  Nothing here
computes any part of the method, and nothing falls back to the CPU: if the
library is not built or there is no CUDA device, calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LYA_LIBRARY may name another build of the same library (the bounds-checked
# one, build(checked=True)); there is no other implementation to fall back to
_LIB_PATH = os.environ.get("LYA_LIBRARY") or os.path.join(_HERE, "_build", "liblya.so")
_lock = threading.Lock()
_lib = None

LYA_OK, LYA_EINVAL, LYA_ENOMEM, LYA_ECUDA, LYA_ENOCONV, LYA_ETIMEDOUT, LYA_EBUDGET, LYA_EDEVICE, LYA_EBUSY = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
SRC_HOST, SRC_DEVICE_COPY, SRC_DEVICE_BORROW = 0, 1, 2
PREC_F32_COMPENSATED, PREC_F32_NAIVE, PREC_F64 = 0, 1, 2
PROFILE_SAMPLED, PROFILE_AVERAGED = 0, 1
EXP_MUFU, EXP_RECURRENCE, EXP_POLY_SPLIT = 0, 1, 2


class LyaError(RuntimeError):
    """A liblya call returned a status other than LYA_OK."""

    def __init__(self, status: int, what: str):
        self.status = status
        msg = load_library().lya_strerror(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")


class _FieldDesc(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("z", ctypes.c_double), ("h", ctypes.c_double),
                ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
                ("omega_b", ctypes.c_double), ("y_he", ctypes.c_double),
                ("n_skewers", ctypes.c_int64), ("n_pix", ctypes.c_int64),
                ("has_temp", ctypes.c_int)]


class _ExtractParams(ctypes.Structure):
    _fields_ = [("t_mode", ctypes.c_int), ("T0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("delta_pivot", ctypes.c_double), ("gamma12", ctypes.c_double),
                ("nsigma", ctypes.c_double), ("precision", ctypes.c_int), ("profile", ctypes.c_int),
                ("exp_method", ctypes.c_int)]


class _FluxStats(ctypes.Structure):
    _fields_ = [("mean_flux", ctypes.c_double), ("var_flux", ctypes.c_double),
                ("tau_eff", ctypes.c_double), ("pdf", ctypes.c_int64 * 21), ("n", ctypes.c_int64)]


class _MockParams(ctypes.Structure):
    _fields_ = [("fwhm_kms", ctypes.c_double), ("bin_kms", ctypes.c_double), ("snr", ctypes.c_double),
                ("max_kms", ctypes.c_double), ("nsigma", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("row0", ctypes.c_int64)]


class _SightlineDesc(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("z", ctypes.c_double), ("h", ctypes.c_double),
                ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double), ("k_j", ctypes.c_double),
                ("sigma_delta", ctypes.c_double), ("k_f", ctypes.c_double), ("seed", ctypes.c_uint64)]


class _MeanFluxIter(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double), ("lo", ctypes.c_double), ("hi", ctypes.c_double), ("g", ctypes.c_double),
                ("iter", ctypes.c_int), ("max_iter", ctypes.c_int), ("done", ctypes.c_int), ("status", ctypes.c_int),
                ("target", ctypes.c_double), ("tol", ctypes.c_double), ("n", ctypes.c_double)]


# int allreduce(double* values, int count, void* user): values summed over all parts, in place
_ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p)


class _ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("step_target_us", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class _ServerResult(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("A", ctypes.c_double),
                ("iterations", ctypes.c_int), ("stats", _FluxStats), ("flux", ctypes.c_void_p),
                ("n_ids", ctypes.c_int64), ("n_pix", ctypes.c_int64), ("t_submit_ns", ctypes.c_uint64),
                ("t_admit_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64)]


class _ServerInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("arena_used", ctypes.c_size_t), ("arena_peak", ctypes.c_size_t),
                ("arena_capacity", ctypes.c_size_t), ("slots_in_use", ctypes.c_int), ("queued", ctypes.c_int),
                ("group_shift", ctypes.c_int * 14)]


def kernel_launches() -> int:
    """Kernels liblya has launched in this process (lya_kernel_launches)."""
    return int(load_library().lya_kernel_launches())


def scratch_high_watermark(reset: bool = False) -> int:
    """Used-memory high watermark (bytes) of the library's scratch pool on the
    current device, then reset it if asked (lya_scratch_high_watermark)."""
    v = ctypes.c_uint64(0)
    _check(load_library().lya_scratch_high_watermark(1 if reset else 0, ctypes.byref(v)),
           "lya_scratch_high_watermark")
    return int(v.value)


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load liblya.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.lya_strerror.argtypes = [i32]
        lib.lya_strerror.restype = ctypes.c_char_p
        lib.lya_version.argtypes = []
        lib.lya_version.restype = ctypes.c_char_p
        lib.lya_kernel_launches.argtypes = []
        lib.lya_kernel_launches.restype = ctypes.c_uint64
        lib.lya_scratch_high_watermark.argtypes = [i32, ctypes.POINTER(ctypes.c_uint64)]
        lib.lya_create_field.argtypes = [ctypes.POINTER(_FieldDesc), vp, vp, vp, i32, vp, ctypes.POINTER(vp)]
        lib.lya_field_load.argtypes = [vp, vp, vp, vp, i32, vp]
        lib.lya_destroy_field.argtypes = [vp]
        lib.lya_field_status.argtypes = [vp, vp]
        lib.lya_field_shape.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.lya_extract_skewers.argtypes = [vp, ctypes.POINTER(_ExtractParams), vp, i64, vp, vp]
        lib.lya_rescale_mean_flux.argtypes = [vp, i64, d, d, i32, ctypes.POINTER(d), vp, vp]
        lib.lya_rescale_mean_flux_noalloc.argtypes = [vp, i64, d, d, i32, ctypes.POINTER(d), vp, vp]
        lib.lya_rescale_mean_flux_stats.argtypes = [vp, i64, d, d, i32, ctypes.POINTER(d), vp,
                                                    ctypes.POINTER(_FluxStats), vp]
        lib.lya_flux_stats.argtypes = [vp, i64, ctypes.POINTER(_FluxStats), vp]
        lib.lya_tau_moments.argtypes = [vp, i64, ctypes.POINTER(d), vp]
        lib.lya_mean_flux_sums.argtypes = [vp, i64, d, ctypes.POINTER(d), vp]
        lib.lya_flux_at.argtypes = [vp, i64, d, vp, vp]
        lib.lya_mean_flux_start.argtypes = [ctypes.POINTER(d), d, d, i32, ctypes.POINTER(_MeanFluxIter)]
        lib.lya_mean_flux_step.argtypes = [ctypes.POINTER(_MeanFluxIter), ctypes.POINTER(d)]
        lib.lya_rescale_mean_flux_sharded.argtypes = [vp, i64, d, d, i32, _ALLREDUCE_FN, vp, ctypes.POINTER(d),
                                                      ctypes.POINTER(i32), vp, vp]
        u64 = ctypes.c_uint64
        lib.lya_field_pixel_width.argtypes = [vp, ctypes.POINTER(d)]
        lib.lya_generate_sightlines.argtypes = [ctypes.POINTER(_SightlineDesc), i64, i64, i64, vp, vp, vp]
        lib.lya_flux_power_3d_shells.argtypes = [i64, i32, ctypes.POINTER(i64)]
        lib.lya_flux_power_3d.argtypes = [vp, vp, i64, i64, i32, d, d, vp, vp, vp, vp, vp]
        lib.lya_mock_shape.argtypes = [i64, d, ctypes.POINTER(_MockParams), ctypes.POINTER(i64)]
        lib.lya_mock_spectra.argtypes = [vp, i64, i64, d, ctypes.POINTER(_MockParams), vp, vp]
        lib.lya_flux_power_1d.argtypes = [vp, i64, i64, d, vp, vp, ctypes.POINTER(d), vp]
        lib.lya_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(vp)]
        lib.lya_server_autotune.argtypes = [vp, vp, ctypes.POINTER(_ExtractParams), i64, ctypes.POINTER(i32)]
        lib.lya_server_submit.argtypes = [vp, vp, ctypes.POINTER(_ExtractParams), vp, i64, d, ctypes.POINTER(u64)]
        lib.lya_server_poll.argtypes = [vp, u64, ctypes.POINTER(_ServerResult)]
        lib.lya_server_wait.argtypes = [vp, u64, d, ctypes.POINTER(_ServerResult)]
        lib.lya_server_copy_flux.argtypes = [vp, u64, vp, vp]
        lib.lya_server_release.argtypes = [vp, u64]
        lib.lya_server_info.argtypes = [vp, ctypes.POINTER(_ServerInfo)]
        lib.lya_server_destroy.argtypes = [vp]
        for name in ("lya_create_field", "lya_field_load", "lya_destroy_field", "lya_field_status",
                     "lya_field_shape", "lya_extract_skewers", "lya_rescale_mean_flux",
                     "lya_rescale_mean_flux_noalloc", "lya_rescale_mean_flux_stats", "lya_flux_stats", "lya_tau_moments",
                     "lya_mean_flux_sums", "lya_flux_at", "lya_mean_flux_start", "lya_mean_flux_step",
                     "lya_rescale_mean_flux_sharded", "lya_server_create", "lya_server_autotune",
                     "lya_server_submit", "lya_server_poll", "lya_server_wait", "lya_server_copy_flux",
                     "lya_server_release", "lya_server_info", "lya_server_destroy", "lya_field_pixel_width",
                     "lya_mock_shape", "lya_mock_spectra", "lya_flux_power_1d", "lya_generate_sightlines",
                     "lya_flux_power_3d_shells", "lya_flux_power_3d"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != LYA_OK:
        raise LyaError(status, what)


def _torch():
    import torch
    return torch


def _stream_handle(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_out_like(ref, out, name, ref_name="tau"):
    """``out`` must hold exactly as many values as ``ref``, on the same device
    (the kernels write ref.numel() values into it)."""
    if out.numel() != ref.numel():
        raise ValueError(f"{name} must have {ref.numel()} elements like {ref_name}, not {out.numel()}")
    if out.device != ref.device:
        raise ValueError(f"{name} is on {out.device} but {ref_name} is on {ref.device}")
    return out


def _on(t):
    """The CUDA device of tensor ``t`` made current for the library call (the
    C ABI works on the current device)."""
    return _torch().cuda.device(t.device)


def _require_cuda_f32(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float32")
    return t


@dataclass
class ExtractParams:
    """Physics of one extraction (Eq. 4-6); see lya_extract_params in include/lya.h."""
    t_mode: int = 0
    T0: float = 1.5e4
    gamma: float = 1.5
    delta_pivot: float = 10.0
    gamma12: float = 1.0
    nsigma: float = 8.0
    precision: int = PREC_F32_COMPENSATED
    profile: int = 0                    # PROFILE_SAMPLED (Eq. 6) or PROFILE_AVERAGED
    exp_method: int = 0                 # EXP_MUFU, EXP_RECURRENCE or EXP_POLY_SPLIT

    def _c(self) -> _ExtractParams:
        return _ExtractParams(int(self.t_mode), float(self.T0), float(self.gamma),
                              float(self.delta_pivot), float(self.gamma12), float(self.nsigma),
                              int(self.precision), int(self.profile), int(self.exp_method))


class Field:
    """A skewer field resident in device memory (lya_create_field).

    ``rho`` (1+delta), ``vpec`` (km/s) and ``temp`` (K, optional) are either
    numpy arrays / CPU tensors (copied from the host) or CUDA tensors (copied,
    or referenced when ``borrow=True``), shaped [n_skewers][n_pix], float32.
    """

    def __init__(self, rho, vpec, temp=None, *, box: float, z: float, h: float = 0.72,
                 omega_m: float = 0.26, omega_l: float = 0.74, omega_b: float = 0.0444,
                 y_he: float = 0.24, borrow: bool = False, stream=None):
        lib = load_library()
        torch = _torch()
        self._handle = None
        self._keep = None
        arrays, src = self._marshal(rho, vpec, temp, borrow)
        S, N = arrays[0].shape
        desc = _FieldDesc(box, z, h, omega_m, omega_l, omega_b, y_he, S, N, 1 if temp is not None else 0)
        out = ctypes.c_void_p()
        ptrs = [self._ptr(a) for a in arrays]
        _check(lib.lya_create_field(ctypes.byref(desc), ptrs[0], ptrs[1], ptrs[2], src,
                                    _stream_handle(stream) if torch.cuda.is_available() else None,
                                    ctypes.byref(out)), "lya_create_field")
        self._handle = out
        # the device the field lives on (the current one at creation)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.n_skewers, self.n_pix = S, N
        self.has_temp = temp is not None
        self.box, self.z = box, z
        if src == SRC_DEVICE_BORROW:
            self._keep = arrays          # the field references these tensors

    @staticmethod
    def _marshal(rho, vpec, temp, borrow):
        torch = _torch()
        if isinstance(rho, torch.Tensor) and rho.is_cuda:
            arrs = [_require_cuda_f32(rho, "rho"), _require_cuda_f32(vpec, "vpec"),
                    None if temp is None else _require_cuda_f32(temp, "temp")]
            src = SRC_DEVICE_BORROW if borrow else SRC_DEVICE_COPY
        else:
            if borrow:
                raise ValueError("borrow=True needs CUDA tensors")
            conv = [None if a is None else np.ascontiguousarray(
                a.numpy() if isinstance(a, torch.Tensor) else a, dtype=np.float32) for a in (rho, vpec, temp)]
            arrs = conv
            src = SRC_HOST
        if arrs[0].ndim != 2 or tuple(arrs[1].shape) != tuple(arrs[0].shape) or (
                arrs[2] is not None and tuple(arrs[2].shape) != tuple(arrs[0].shape)):
            raise ValueError("rho, vpec and temp must share a 2-D shape [n_skewers][n_pix]")
        return arrs, src

    @staticmethod
    def _ptr(a):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            return a.ctypes.data
        return a.data_ptr()

    def load(self, rho, vpec, temp=None, stream=None):
        """Overwrite the field's arrays (lya_field_load)."""
        arrays, src = self._marshal(rho, vpec, temp, False)
        ptrs = [self._ptr(a) for a in arrays]
        _check(load_library().lya_field_load(self._handle, ptrs[0], ptrs[1], ptrs[2], src,
                                             _stream_handle(stream)), "lya_field_load")

    def status(self, stream=None):
        """Raise if an extraction saw an out-of-range skewer id (lya_field_status)."""
        _check(load_library().lya_field_status(self._handle, _stream_handle(stream)), "lya_field_status")

    @property
    def handle(self):
        return self._handle

    def close(self):
        if self._handle:
            load_library().lya_destroy_field(self._handle)
            self._handle = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def extract_skewers(field: Field, params: ExtractParams, ids=None, out=None, stream=None):
    """tau [n_ids][n_pix] on the device (lya_extract_skewers).

    ``ids``: None (all skewers) or an int64 tensor / array of skewer ids.
    """
    torch = _torch()
    lib = load_library()
    if ids is None:
        n_ids, ids_ptr = field.n_skewers, None
    else:
        ids_t = torch.as_tensor(ids, dtype=torch.int64).to(field.device).contiguous()
        n_ids, ids_ptr = ids_t.numel(), ids_t.data_ptr()
    if out is None:
        out = torch.empty((n_ids, field.n_pix), dtype=torch.float32, device=field.device)
    else:
        _require_cuda_f32(out, "out")
        if out.numel() != n_ids * field.n_pix:
            raise ValueError("out has the wrong size")
        if out.device != field.device:
            raise ValueError(f"out is on {out.device} but the field is on {field.device}")
    p = params._c()
    with torch.cuda.device(field.device):
        _check(lib.lya_extract_skewers(field.handle, ctypes.byref(p), ids_ptr, n_ids,
                                       out.data_ptr() if n_ids else None, _stream_handle(stream)),
               "lya_extract_skewers")
    if ids is not None:
        out._lya_ids = ids_t            # keep the id buffer alive until the kernel ran
    return out


def rescale_mean_flux(tau, target: float, tol: float = 1e-12, max_iter: int = 50,
                      flux_out=True, stream=None):
    """Mean-flux rescaling (lya_rescale_mean_flux): returns (A, F or None)."""
    torch = _torch()
    _require_cuda_f32(tau, "tau")
    F = None
    if flux_out is True:
        F = torch.empty_like(tau)
    elif flux_out is not None and flux_out is not False:
        F = _check_out_like(tau, _require_cuda_f32(flux_out, "flux_out"), "flux_out")
    A = ctypes.c_double(math.nan)
    with _on(tau):
        _check(load_library().lya_rescale_mean_flux(tau.data_ptr(), tau.numel(), float(target), float(tol),
                                                    int(max_iter), ctypes.byref(A),
                                                    F.data_ptr() if F is not None else None,
                                                    _stream_handle(stream)), "lya_rescale_mean_flux")
    return A.value, F


def rescale_mean_flux_stats(tau, target: float, tol: float = 1e-12, max_iter: int = 50, flux_out=True,
                            stream=None):
    """lya_rescale_mean_flux_stats: (A, F or None, FluxStats) with the statistics
    gathered in the root-find's final flux pass."""
    torch = _torch()
    _require_cuda_f32(tau, "tau")
    F = None
    if flux_out is True:
        F = torch.empty_like(tau)
    elif flux_out is not None and flux_out is not False:
        F = _check_out_like(tau, _require_cuda_f32(flux_out, "flux_out"), "flux_out")
    A = ctypes.c_double(math.nan)
    out = _FluxStats()
    with _on(tau):
        _check(load_library().lya_rescale_mean_flux_stats(tau.data_ptr(), tau.numel(), float(target), float(tol),
                                                          int(max_iter), ctypes.byref(A),
                                                          F.data_ptr() if F is not None else None,
                                                          ctypes.byref(out), _stream_handle(stream)),
               "lya_rescale_mean_flux_stats")
    st = FluxStats(out.mean_flux, out.var_flux, out.tau_eff, np.array(out.pdf[:], dtype=np.int64), out.n)
    return A.value, F, st


def rescale_mean_flux_noalloc(tau, target: float, flux_out, tol: float = 1e-12, max_iter: int = 50,
                              stream=None):
    """lya_rescale_mean_flux_noalloc: the root-find with no device allocation.

    ``flux_out`` is a caller-provided CUDA float32 tensor shaped like ``tau``
    (or None); the library allocates nothing.  Returns A.
    """
    _require_cuda_f32(tau, "tau")
    if flux_out is not None:
        _check_out_like(tau, _require_cuda_f32(flux_out, "flux_out"), "flux_out")
    A = ctypes.c_double(math.nan)
    with _on(tau):
        _check(load_library().lya_rescale_mean_flux_noalloc(
            tau.data_ptr(), tau.numel(), float(target), float(tol), int(max_iter), ctypes.byref(A),
            flux_out.data_ptr() if flux_out is not None else None, _stream_handle(stream)),
            "lya_rescale_mean_flux_noalloc")
    return A.value


def tau_moments(tau, stream=None):
    """(sum tau, number of zeros, number of invalid values) of device values (lya_tau_moments)."""
    _require_cuda_f32(tau, "tau")
    out = (ctypes.c_double * 3)()
    with _on(tau):
        _check(load_library().lya_tau_moments(tau.data_ptr(), tau.numel(), out, _stream_handle(stream)),
               "lya_tau_moments")
    return tuple(out)


def mean_flux_sums(tau, A: float, stream=None):
    """(sum e, sum tau e, sum tau^2 e), e = exp(-A tau), over device values (lya_mean_flux_sums)."""
    _require_cuda_f32(tau, "tau")
    out = (ctypes.c_double * 3)()
    with _on(tau):
        _check(load_library().lya_mean_flux_sums(tau.data_ptr(), tau.numel(), float(A), out,
                                                 _stream_handle(stream)), "lya_mean_flux_sums")
    return tuple(out)


def flux_at(tau, A: float, out=None, stream=None):
    """F = exp(-A tau) on the device for a given A (lya_flux_at)."""
    _require_cuda_f32(tau, "tau")
    F = out if out is not None else _torch().empty_like(tau)
    _check_out_like(tau, _require_cuda_f32(F, "out"), "out")
    with _on(tau):
        _check(load_library().lya_flux_at(tau.data_ptr(), tau.numel(), float(A), F.data_ptr(),
                                          _stream_handle(stream)), "lya_flux_at")
    return F


class MeanFluxIter:
    """The Sec. 2.3 iteration of a split request, stepped by the library on
    the host (lya_mean_flux_iter): ``A``, ``done``, ``status``, ``iter``, ``g``."""

    def __init__(self, c: _MeanFluxIter):
        self._c = c

    def __getattr__(self, name):
        return getattr(self._c, name)


def mean_flux_start(totals, target: float, tol: float = 1e-12, max_iter: int = 50) -> MeanFluxIter:
    """lya_mean_flux_start from totals = (sum tau, zeros, invalid, n) over all
    parts.  Raises LyaError when the iteration cannot start."""
    it = _MeanFluxIter()
    t = (ctypes.c_double * 4)(*[float(x) for x in totals])
    _check(load_library().lya_mean_flux_start(t, float(target), float(tol), int(max_iter), ctypes.byref(it)),
           "lya_mean_flux_start")
    return MeanFluxIter(it)


def mean_flux_step(it: MeanFluxIter, sums) -> bool:
    """lya_mean_flux_step with sums = (sum e, sum tau e, sum tau^2 e) at it.A
    over all parts; returns True once the iteration has ended.  Raises
    LyaError if it ended without converging."""
    v = (ctypes.c_double * 3)(*[float(x) for x in sums])
    _check(load_library().lya_mean_flux_step(ctypes.byref(it._c), v), "lya_mean_flux_step")
    return bool(it.done)


def rescale_mean_flux_sharded(tau, target: float, allreduce, tol: float = 1e-12, max_iter: int = 50,
                              flux_out=True, stream=None):
    """lya_rescale_mean_flux_sharded: this part's tau (CUDA tensor, may be
    empty) and ``allreduce(list_of_floats) -> list_of_floats`` summing over
    all parts.  Returns (A, steps, F of this part or None)."""
    torch = _torch()
    _require_cuda_f32(tau, "tau")
    F = None
    if flux_out is True:
        F = torch.empty_like(tau)
    elif flux_out is not None and flux_out is not False:
        F = _check_out_like(tau, _require_cuda_f32(flux_out, "flux_out"), "flux_out")
    errors = []

    def cb(ptr, count, _user):
        try:
            out = allreduce([ptr[k] for k in range(count)])
            for k in range(count):
                ptr[k] = float(out[k])
            return 0
        except Exception as exc:             # surfaced after the call
            errors.append(exc)
            return 1

    fn = _ALLREDUCE_FN(cb)
    A = ctypes.c_double(math.nan)
    it = ctypes.c_int(0)
    with _on(tau):
        status = load_library().lya_rescale_mean_flux_sharded(
            tau.data_ptr() if tau.numel() else None, tau.numel(), float(target), float(tol), int(max_iter), fn,
            None, ctypes.byref(A), ctypes.byref(it), F.data_ptr() if (F is not None and tau.numel()) else None,
            _stream_handle(stream))
    if errors:
        raise errors[0]
    _check(status, "lya_rescale_mean_flux_sharded")
    return A.value, it.value, F


@dataclass
class FluxStats:
    mean_flux: float
    var_flux: float
    tau_eff: float
    pdf: np.ndarray
    n: int


def flux_stats(flux, stream=None) -> FluxStats:
    """<F>, Var F, tau_eff, 21-bin PDF of device flux values (lya_flux_stats)."""
    _require_cuda_f32(flux, "flux")
    out = _FluxStats()
    with _on(flux):
        _check(load_library().lya_flux_stats(flux.data_ptr(), flux.numel(), ctypes.byref(out),
                                             _stream_handle(stream)), "lya_flux_stats")
    return FluxStats(out.mean_flux, out.var_flux, out.tau_eff, np.array(out.pdf[:], dtype=np.int64), out.n)


@dataclass
class ServerResult:
    """State of one served request (lya_server_result)."""
    done: bool
    status: int
    A: float
    iterations: int
    stats: FluxStats
    n_ids: int
    n_pix: int
    t_submit_ns: int
    t_admit_ns: int
    t_done_ns: int
    flux_ptr: int

    @property
    def latency_s(self) -> float:
        return (self.t_done_ns - self.t_submit_ns) * 1e-9 if self.done else math.nan


class Server:
    """The serving loop (lya_server_*): requests are queued with ``submit``,
    admitted by memory budget and run in steps by the library's worker thread.

    ``budget_bytes`` bounds tau + F of admitted requests (8 bytes per pixel);
    ``max_slots`` the requests in flight; ``step_target_us`` the optical-depth
    work packed into one step.
    """

    def __init__(self, budget_bytes: int, max_slots: int = 256, step_target_us: float = 2000.0,
                 tol: float = 1e-12, max_iter: int = 50):
        lib = load_library()
        self._handle = None
        cfg = _ServerConfig(int(budget_bytes), int(max_slots), float(step_target_us), float(tol), int(max_iter))
        out = ctypes.c_void_p()
        _check(lib.lya_server_create(ctypes.byref(cfg), ctypes.byref(out)), "lya_server_create")
        self._handle = out
        self._fields = {}                # keep fields of unfinished requests alive

    def autotune(self, field: Field, params: ExtractParams, max_rows: int = 1024) -> int:
        """Choose the group shape for this field's skewer length; returns log2(skewers per CTA)."""
        shift = ctypes.c_int(-1)
        p = params._c()
        _check(load_library().lya_server_autotune(self._handle, field.handle, ctypes.byref(p), int(max_rows),
                                                  ctypes.byref(shift)), "lya_server_autotune")
        return shift.value

    def submit(self, field: Field, params: ExtractParams, ids, target_mean_flux: float) -> int:
        ids_h = np.ascontiguousarray(np.asarray(ids, dtype=np.int64).ravel())
        ticket = ctypes.c_uint64()
        p = params._c()
        _check(load_library().lya_server_submit(self._handle, field.handle, ctypes.byref(p), ids_h.ctypes.data,
                                                ids_h.size, float(target_mean_flux), ctypes.byref(ticket)),
               "lya_server_submit")
        self._fields[ticket.value] = field
        return ticket.value

    @staticmethod
    def _result(r: _ServerResult) -> ServerResult:
        st = FluxStats(r.stats.mean_flux, r.stats.var_flux, r.stats.tau_eff,
                       np.array(r.stats.pdf[:], dtype=np.int64), r.stats.n)
        return ServerResult(bool(r.done), int(r.status), r.A, int(r.iterations), st, int(r.n_ids), int(r.n_pix),
                            int(r.t_submit_ns), int(r.t_admit_ns), int(r.t_done_ns), int(r.flux or 0))

    def poll(self, ticket: int) -> ServerResult:
        r = _ServerResult()
        _check(load_library().lya_server_poll(self._handle, int(ticket), ctypes.byref(r)), "lya_server_poll")
        return self._result(r)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> ServerResult:
        r = _ServerResult()
        _check(load_library().lya_server_wait(self._handle, int(ticket), float(timeout_s), ctypes.byref(r)),
               "lya_server_wait")
        return self._result(r)

    def flux(self, ticket: int, out=None, stream=None):
        """A copy of a finished request's F as a CUDA tensor [n_ids][n_pix]."""
        torch = _torch()
        r = self.poll(ticket)
        if out is None:
            out = torch.empty((r.n_ids, r.n_pix), dtype=torch.float32, device="cuda")
        _require_cuda_f32(out, "out")
        if out.numel() != r.n_ids * r.n_pix:
            raise ValueError("out has the wrong size")
        _check(load_library().lya_server_copy_flux(self._handle, int(ticket), out.data_ptr(),
                                                   _stream_handle(stream)), "lya_server_copy_flux")
        return out

    def release(self, ticket: int):
        _check(load_library().lya_server_release(self._handle, int(ticket)), "lya_server_release")
        self._fields.pop(int(ticket), None)

    def info(self) -> dict:
        i = _ServerInfo()
        _check(load_library().lya_server_info(self._handle, ctypes.byref(i)), "lya_server_info")
        return {"steps": i.steps, "submitted": i.submitted, "completed": i.completed, "failed": i.failed,
                "arena_used": i.arena_used, "arena_peak": i.arena_peak, "arena_capacity": i.arena_capacity,
                "slots_in_use": i.slots_in_use, "queued": i.queued, "group_shift": list(i.group_shift)}

    def close(self):
        if self._handle:
            load_library().lya_server_destroy(self._handle)
            self._handle = None
            self._fields.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class MockParams:
    """Instrument processing of mock spectra (Sec. 4); see lya_mock_params in include/lya.h."""
    fwhm_kms: float = 0.0
    bin_kms: float = 0.0
    snr: float = 0.0
    max_kms: float = 0.0
    nsigma: float = 6.0
    seed: int = 0
    row0: int = 0

    def _c(self) -> _MockParams:
        return _MockParams(float(self.fwhm_kms), float(self.bin_kms), float(self.snr), float(self.max_kms),
                           float(self.nsigma), int(self.seed) & 0xFFFFFFFFFFFFFFFF, int(self.row0))


def field_pixel_width(field: Field) -> float:
    """Pixel velocity width of the field's skewers, km/s (lya_field_pixel_width)."""
    du = ctypes.c_double()
    _check(load_library().lya_field_pixel_width(field.handle, ctypes.byref(du)), "lya_field_pixel_width")
    return du.value


def mock_shape(n_pix: int, du_kms: float, params: MockParams) -> int:
    n = ctypes.c_int64()
    p = params._c()
    _check(load_library().lya_mock_shape(int(n_pix), float(du_kms), ctypes.byref(p), ctypes.byref(n)),
           "lya_mock_shape")
    return n.value


def mock_spectra(flux, du_kms: float, params: MockParams, out=None, stream=None):
    """Mock spectra [n_skewers][n_out] on the device (lya_mock_spectra)."""
    torch = _torch()
    _require_cuda_f32(flux, "flux")
    if flux.dim() != 2:
        raise ValueError("flux must be [n_skewers][n_pix]")
    S, N = flux.shape
    M = mock_shape(N, du_kms, params)
    if out is None:
        out = torch.empty((S, M), dtype=torch.float32, device=flux.device)
    _require_cuda_f32(out, "out")
    if out.numel() != S * M:
        raise ValueError("out has the wrong size")
    p = params._c()
    _check(load_library().lya_mock_spectra(flux.data_ptr(), S, N, float(du_kms), ctypes.byref(p), out.data_ptr(),
                                           _stream_handle(stream)), "lya_mock_spectra")
    return out


def flux_power_1d(flux, du_kms: float, stream=None):
    """(k [s/km], P(k) [km/s], <F>) of the line-of-sight flux contrast (lya_flux_power_1d)."""
    _require_cuda_f32(flux, "flux")
    if flux.dim() != 2:
        raise ValueError("flux must be [n_skewers][n_pix]")
    S, N = flux.shape
    k = np.empty(N // 2 + 1)
    P = np.empty(N // 2 + 1)
    mean = ctypes.c_double()
    _check(load_library().lya_flux_power_1d(flux.data_ptr(), S, N, float(du_kms), k.ctypes.data, P.ctypes.data,
                                            ctypes.byref(mean), _stream_handle(stream)), "lya_flux_power_1d")
    return k, P, mean.value


def generate_sightlines(n_pix: int, first_id: int, n_ids: int, *, box: float, z: float, k_j: float,
                        sigma_delta: float, seed: int, k_f: float = 0.0, h: float = 0.72, omega_m: float = 0.26,
                        omega_l: float = 0.74, rho_out=None, vpec_out=None, stream=None):
    """(1 + delta, v_pec) [n_ids][n_pix] generated on the device (lya_generate_sightlines)."""
    torch = _torch()
    if rho_out is None:
        rho_out = torch.empty((n_ids, n_pix), dtype=torch.float32, device="cuda")
    if vpec_out is None:
        vpec_out = torch.empty((n_ids, n_pix), dtype=torch.float32, device="cuda")
    for t, name in ((rho_out, "rho_out"), (vpec_out, "vpec_out")):
        _require_cuda_f32(t, name)
        if t.numel() != n_ids * n_pix:
            raise ValueError(f"{name} has the wrong size")
    desc = _SightlineDesc(float(box), float(z), float(h), float(omega_m), float(omega_l), float(k_j),
                          float(sigma_delta), float(k_f), int(seed) & 0xFFFFFFFFFFFFFFFF)
    _check(load_library().lya_generate_sightlines(ctypes.byref(desc), int(n_pix), int(first_id), int(n_ids),
                                                  rho_out.data_ptr(), vpec_out.data_ptr(), _stream_handle(stream)),
           "lya_generate_sightlines")
    return rho_out, vpec_out


def flux_power_3d(flux, cells, n_perp: int, box: float, noise_sigma: float = 0.0, stream=None):
    """Shell-averaged Eq. 7 3D flux power of lines of sight (lya_flux_power_3d).

    ``cells``: transverse cell of each line, ix * n_perp + iy (or an [n][2]
    array of (ix, iy)).  Returns (k_mean, P_true, P_box, n_modes) numpy arrays.
    """
    _require_cuda_f32(flux, "flux")
    if flux.dim() != 2:
        raise ValueError("flux must be [n_los][n_pix]")
    S, N = flux.shape
    c = np.asarray(cells, dtype=np.int64)
    if c.ndim == 2:
        c = c[:, 0] * n_perp + c[:, 1]
    c = np.ascontiguousarray(c.ravel(), dtype=np.int32)
    if c.size != S:
        raise ValueError("one cell per line of sight")
    lib = load_library()
    ns = ctypes.c_int64()
    _check(lib.lya_flux_power_3d_shells(N, int(n_perp), ctypes.byref(ns)), "lya_flux_power_3d_shells")
    k, pt, pb, nm = (np.zeros(ns.value) for _ in range(4))
    _check(lib.lya_flux_power_3d(flux.data_ptr(), c.ctypes.data, S, N, int(n_perp), float(box), float(noise_sigma),
                                 k.ctypes.data, pt.ctypes.data, pb.ctypes.data, nm.ctypes.data,
                                 _stream_handle(stream)), "lya_flux_power_3d")
    return k, pt, pb, nm
