"""FP64 CPU oracle for Lyman-alpha optical-depth extraction (test infrastructure).

This package is the plain, slow reference that the CUDA path is checked
against.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product package never does.  It shares
no code with the CUDA path: the arithmetic lives in ``lya_oracle.c`` (plain C,
FP64, OpenMP over skewers) and this module only marshals numpy arrays.

Functions follow Greig, Bolton & Wyithe (2011):
  * :func:`tau`          -- Eq. 4-6, the full periodic O(N^2) sum (Sec. 2.3)
  * :func:`rescale`      -- mean-flux normalisation A (Sec. 2.3)
  * :func:`flux`         -- F = exp(-A tau) (Sec. 2.3)
  * :func:`flux_stats`   -- <F>, Var F, tau_eff = -ln<F>, 21-bin PDF (Sec. 5.2)
  * :func:`pdf_bin`      -- the PDF bin of one value (Sec. 5.2)
plus the unit helpers (H(z), pixel widths, nbar_H, b(T), n_HI) they use.
The mock-spectrum processing of Sec. 4 and the 1D flux power spectrum of
Sec. 5.3 are in :mod:`oracle.mock` (FP64 numpy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lya_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblya_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``lya_oracle.c`` into ``_build/liblya_oracle.so`` with gcc.

    Plain ``-O2``, no fast-math (the oracle must round like IEEE FP64), and
    OpenMP for the loop over skewers.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double), ("z", ctypes.c_double), ("h", ctypes.c_double),
        ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
        ("omega_b", ctypes.c_double), ("y_he", ctypes.c_double),
        ("t_mode", ctypes.c_int), ("T0", ctypes.c_double), ("gamma", ctypes.c_double),
        ("delta_pivot", ctypes.c_double), ("gamma12", ctypes.c_double),
        ("profile", ctypes.c_int),
    ]


@dataclass
class Params:
    """Physical parameters of one extraction (defaults: the paper's cosmology, Sec. 2).

    ``t_mode`` 0 takes T per pixel from the input array; 1 uses Eq. 5,
    T = T0 (1+delta)^(gamma-1) with T held constant above 1+delta = delta_pivot.
    ``profile`` 1 averages each line's Gaussian over the pixel's velocity cell
    instead of sampling it at the pixel's velocity (Eq. 6 as written).
    """
    box: float = 20.0           # h^-1 Mpc
    z: float = 2.5
    h: float = 0.72
    omega_m: float = 0.26
    omega_l: float = 0.74
    omega_b: float = 0.0444
    y_he: float = 0.24
    t_mode: int = 0
    T0: float = 1.5e4
    gamma: float = 1.5
    delta_pivot: float = 10.0
    gamma12: float = 1.0
    profile: int = 0            # 0: Eq. 6 sampled at v_H(i); 1: averaged over the pixel cell

    def _c(self) -> _Params:
        return _Params(self.box, self.z, self.h, self.omega_m, self.omega_l,
                       self.omega_b, self.y_he, int(self.t_mode), self.T0,
                       self.gamma, self.delta_pivot, self.gamma12, int(self.profile))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # LYA_ORACLE_LIB lets the mutation tests load a deliberately broken
            # build of lya_oracle.c to show that the pins catch it.
            path = os.environ.get("LYA_ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            P = ctypes.POINTER(_Params)
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            fp = ctypes.POINTER(ctypes.c_float)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_int64)
            for name in ("orc_hubble", "orc_mean_nh"):
                getattr(lib, name).argtypes = [P]
                getattr(lib, name).restype = d
            for name in ("orc_pixel_proper_cm", "orc_pixel_velocity"):
                getattr(lib, name).argtypes = [P, i64]
                getattr(lib, name).restype = d
            lib.orc_temperature.argtypes = [P, d, d]
            lib.orc_temperature.restype = d
            lib.orc_doppler_b.argtypes = [d]
            lib.orc_doppler_b.restype = d
            lib.orc_nhi.argtypes = [P, d, d]
            lib.orc_nhi.restype = d
            lib.orc_tau.argtypes = [P, i64, i64, fp, fp, fp, dp]
            lib.orc_tau.restype = i32
            lib.orc_rescale.argtypes = [dp, i64, d, d, i32, dp, ctypes.POINTER(i32)]
            lib.orc_rescale.restype = i32
            lib.orc_flux.argtypes = [dp, i64, d, dp]
            lib.orc_flux.restype = None
            lib.orc_pdf_bin.argtypes = [d]
            lib.orc_pdf_bin.restype = i32
            lib.orc_flux_stats_f32.argtypes = [fp, i64, dp, dp, dp, lp]
            lib.orc_flux_stats_f32.restype = i32
            lib.orc_flux_stats_f64.argtypes = [dp, i64, dp, dp, dp, lp]
            lib.orc_flux_stats_f64.restype = i32
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = i32
            _lib = lib
    return _lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- unit helpers (Sec. 2.3) ------------------------------------------------
def hubble(p: Params) -> float:
    """H(z) in km/s/Mpc."""
    return _load().orc_hubble(ctypes.byref(p._c()))


def pixel_velocity(p: Params, n_pix: int) -> float:
    """Hubble-velocity width of one pixel, km/s."""
    return _load().orc_pixel_velocity(ctypes.byref(p._c()), int(n_pix))


def pixel_proper_cm(p: Params, n_pix: int) -> float:
    """Proper pixel width dR of Eq. 6, cm."""
    return _load().orc_pixel_proper_cm(ctypes.byref(p._c()), int(n_pix))


def mean_nh(p: Params) -> float:
    """Mean total hydrogen density nbar_H of Eq. 4, proper cm^-3."""
    return _load().orc_mean_nh(ctypes.byref(p._c()))


def temperature(p: Params, rho: float, t_given: float = 0.0) -> float:
    """Eq. 5 with the pivot (power-law mode) or the given T (stored mode)."""
    return _load().orc_temperature(ctypes.byref(p._c()), float(rho), float(t_given))


def doppler_b(T: float) -> float:
    """b = sqrt(2 k_B T / m_H) in km/s."""
    return _load().orc_doppler_b(float(T))


def nhi(p: Params, rho: float, T: float) -> float:
    """Eq. 4, cm^-3."""
    return _load().orc_nhi(ctypes.byref(p._c()), float(rho), float(T))


def num_threads() -> int:
    """OpenMP threads the oracle's tau loop uses."""
    return int(_load().orc_num_threads())


# ---- the path -----------------------------------------------------------------
def tau(p: Params, rho, vpec, temp=None) -> np.ndarray:
    """Eq. 6 optical depth for skewers [S][N] (FP32 inputs, FP64 result).

    ``rho`` is 1+delta, ``vpec`` the peculiar velocity in km/s, ``temp`` the
    temperature in K (required in stored mode, ignored in power-law mode).
    """
    rho = np.atleast_2d(rho)
    S, N = rho.shape
    r, rp = _f32(rho)
    v, vp = _f32(np.atleast_2d(vpec))
    if v.shape != r.shape:
        raise ValueError("vpec shape differs from rho shape")
    tp = None
    if temp is not None:
        t, tp = _f32(np.atleast_2d(temp))
        if t.shape != r.shape:
            raise ValueError("temp shape differs from rho shape")
    elif p.t_mode == 0:
        raise ValueError("stored-temperature mode needs temp")
    out = np.empty((S, N), dtype=np.float64)
    rc = _load().orc_tau(ctypes.byref(p._c()), S, N, rp, vp, tp,
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError(f"orc_tau failed ({rc})")
    return out


class NoConvergence(RuntimeError):
    pass


def rescale(tau_values, target_mean_flux: float, tol: float = 1e-12,
            max_iter: int = 100):
    """Mean-flux rescaling: A with <exp(-A tau)> = target (Sec. 2.3).

    Returns ``(A, iterations)``.
    """
    t, tp = _f64(np.ravel(tau_values))
    A = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    rc = _load().orc_rescale(tp, t.size, float(target_mean_flux), float(tol),
                             int(max_iter), ctypes.byref(A), ctypes.byref(it))
    if rc == -4:
        raise NoConvergence(f"no A reaches <F> = {target_mean_flux}")
    if rc != 0:
        raise ValueError(f"orc_rescale rejected its input ({rc})")
    return A.value, it.value


def flux(tau_values, A: float) -> np.ndarray:
    """F = exp(-A tau) in FP64."""
    t, tp = _f64(tau_values)
    out = np.empty_like(t)
    _load().orc_flux(tp, t.size, float(A), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def pdf_bin(F: float) -> int:
    """Sec. 5.2 PDF bin of one flux value."""
    return int(_load().orc_pdf_bin(float(F)))


@dataclass
class FluxStats:
    mean_flux: float
    var_flux: float
    tau_eff: float
    pdf: np.ndarray
    n: int


def flux_stats(F) -> FluxStats:
    """<F>, population Var F, tau_eff = -ln<F> and the 21-bin PDF (Sec. 5.2).

    FP32 input is binned exactly (the bin decision is exact for FP32 values);
    FP64 input is binned in FP64.
    """
    F = np.ravel(F)
    mean, var, te = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    pdf = np.zeros(21, dtype=np.int64)
    pp = pdf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if F.dtype == np.float32:
        a, ap = _f32(F)
        rc = _load().orc_flux_stats_f32(ap, a.size, ctypes.byref(mean), ctypes.byref(var),
                                        ctypes.byref(te), pp)
    else:
        a, ap = _f64(F)
        rc = _load().orc_flux_stats_f64(ap, a.size, ctypes.byref(mean), ctypes.byref(var),
                                        ctypes.byref(te), pp)
    if rc != 0:
        raise ValueError("flux_stats needs at least one value")
    return FluxStats(mean.value, var.value, te.value, pdf, int(F.size))
