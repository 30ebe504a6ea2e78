"""Seeded synthetic skewer fields (input generation only).

This module feeds BOTH the FP64 oracle and the CUDA path with identical FP32
inputs.  It holds none of the optical-depth arithmetic: it only draws a
Gaussian random field per skewer and derives the three input arrays the
method consumes (1+delta, the peculiar velocity, and a stored temperature).

Recipe (stands in for the paper's simulated boxes, Sec. 2.1-2.2 and Sec. 4):
  * skewer ``i`` of a field with seed ``s`` draws its Fourier amplitudes from
    ``np.random.default_rng(SeedSequence([s, i]))``, so any subset of skewers
    is reproducible on its own;
  * 1D linear power P(k) ~ k^-1 exp(-(k/k_J)^2) on the modes k_n = 2 pi n / L,
    n = 1 .. N/2-1 (k = 0 and the Nyquist mode are zero), scaled so that
    sum_n P(k_n) = sigma_delta^2 (the ensemble variance of delta);
  * the linear velocity of Eq. 3 in one dimension, v_k = i f aH delta_k / k
    with f = 1 and aH = H(z)/(1+z) in km/s per h^-1 Mpc;
  * the lognormal density 1+delta = exp(delta - sigma_delta^2/2), which stands
    in for the paper's rank-ordered mapping to a hydrodynamical simulation;
  * a stored temperature T = T0 (1+delta)^(gamma-1) (no pivot: the pivot is
    applied by the method itself in its power-law mode).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class FieldSpec:
    """One family of seeded skewers.  Lengths in h^-1 Mpc, k in h Mpc^-1."""
    n_pix: int
    box: float
    z: float
    k_j: float
    sigma_delta: float
    T0: float
    gamma: float
    seed: int
    h: float = 0.72
    omega_m: float = 0.26
    omega_l: float = 0.74

    def with_(self, **kw) -> "FieldSpec":
        return replace(self, **kw)


def hubble_velocity_per_length(spec: FieldSpec) -> float:
    """aH in km/s per comoving h^-1 Mpc, used to scale the linear velocity."""
    e = np.sqrt(spec.omega_m * (1.0 + spec.z) ** 3 + spec.omega_l)
    return 100.0 * e / (1.0 + spec.z)


def _power(spec: FieldSpec) -> tuple[np.ndarray, np.ndarray]:
    n = np.arange(1, spec.n_pix // 2, dtype=np.float64)
    k = 2.0 * np.pi * n / spec.box
    p = np.exp(-(k / spec.k_j) ** 2) / k
    p *= spec.sigma_delta ** 2 / p.sum()
    return k, p


def gaussian_modes(spec: FieldSpec, ids) -> np.ndarray:
    """Unit complex normal amplitudes, one row per skewer id, seeded per id."""
    ids = np.asarray(ids, dtype=np.int64).ravel()
    m = spec.n_pix // 2 - 1
    out = np.empty((ids.size, m), dtype=np.complex128)
    for row, sid in enumerate(ids):
        rng = np.random.default_rng(np.random.SeedSequence([int(spec.seed), int(sid)]))
        g = rng.standard_normal(2 * m)
        out[row].real = g[:m]
        out[row].imag = g[m:]
    return out


def skewers(spec: FieldSpec, ids, with_temp: bool = True, chunk: int = 4096):
    """FP32 arrays (rho = 1+delta, vpec [km/s], temp [K] or None), shape [len(ids)][N]."""
    ids = np.asarray(ids, dtype=np.int64).ravel()
    N = spec.n_pix
    if N < 4 or N % 2:
        raise ValueError("n_pix must be even and >= 4")
    k, p = _power(spec)
    amp = np.sqrt(p)
    ah = hubble_velocity_per_length(spec)
    rho = np.empty((ids.size, N), dtype=np.float32)
    vpec = np.empty((ids.size, N), dtype=np.float32)
    temp = np.empty((ids.size, N), dtype=np.float32) if with_temp else None
    for lo in range(0, ids.size, chunk):
        sub = ids[lo:lo + chunk]
        z = gaussian_modes(spec, sub)
        X = np.zeros((sub.size, N // 2 + 1), dtype=np.complex128)
        # delta(x) = sum_n (a_n cos k_n x + b_n sin k_n x), a, b ~ N(0, P_n)
        X[:, 1:N // 2] = 0.5 * N * np.conj(z) * amp
        delta = np.fft.irfft(X, n=N, axis=1)
        V = np.zeros_like(X)
        V[:, 1:N // 2] = 1j * ah * X[:, 1:N // 2] / k
        v = np.fft.irfft(V, n=N, axis=1)
        r = np.exp(delta - 0.5 * spec.sigma_delta ** 2)
        rho[lo:lo + sub.size] = r
        vpec[lo:lo + sub.size] = v
        if with_temp:
            temp[lo:lo + sub.size] = spec.T0 * r ** (spec.gamma - 1.0)
    return rho, vpec, temp


def random_subset(n_total: int, n_pick: int, seed: int) -> np.ndarray:
    """Sorted random subset of skewer ids (without replacement)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=min(n_pick, n_total), replace=False))


# ---- the workloads of the paper's scale (names say what they are) ----------
# 64 x 256 px, 20 h^-1 Mpc box at z = 2.5: the oracle finishes it in seconds.
TINY_20MPC = FieldSpec(n_pix=256, box=20.0, z=2.5, k_j=10.0, sigma_delta=1.0,
                       T0=1.5e4, gamma=1.5, seed=0)
TINY_20MPC_SKEWERS = 64
TINY_20MPC_FT = 0.80

# 65,536 x 4,096 px from a periodic 1 h^-1 Gpc box at z = 2.5 (pixel 0.244
# h^-1 Mpc, near the Jeans scale), the scale of the paper's large volumes.
GPC_4096 = FieldSpec(n_pix=4096, box=1000.0, z=2.5, k_j=4.0, sigma_delta=1.5,
                     T0=1.5e4, gamma=1.5, seed=1)
GPC_4096_SKEWERS = 65536
GPC_4096_FT = 0.80
GPC_4096_ORACLE_SUBSET = (256, 1001)       # (count, rng seed)
GPC_4096_PRECISION_SUBSET = (1024, 1002)

# Rows along the contiguous axis of a periodic 1536^3 grid, 1 h^-1 Gpc box at z = 2.3.
GRID_1536 = FieldSpec(n_pix=1536, box=1000.0, z=2.3, k_j=4.0, sigma_delta=1.5,
                      T0=2.0e4, gamma=1.4, seed=4)
GRID_1536_ROWS = 1536 * 1536
GRID_1536_FT = 0.78
GRID_1536_ORACLE_SUBSET = (512, 1004)


def _skewers_chunk(args):
    spec, ids, with_temp = args
    return skewers(spec, ids, with_temp=with_temp)


def skewers_parallel(spec: FieldSpec, ids, with_temp: bool = True, workers: int | None = None,
                     chunk: int = 2048):
    """Same arrays as :func:`skewers`, generated by a spawn-started process pool.

    Spawned workers re-import the caller's main module, so a script calling
    this must keep its top-level work under ``if __name__ == "__main__":``.
    A worker that dies raises BrokenProcessPool here instead of hanging.
    """
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    ids = np.asarray(ids, dtype=np.int64).ravel()
    workers = workers or max(1, min(16, (os.cpu_count() or 1)))
    if workers == 1 or ids.size <= chunk:
        return skewers(spec, ids, with_temp=with_temp)
    N = spec.n_pix
    rho = np.empty((ids.size, N), dtype=np.float32)
    vpec = np.empty((ids.size, N), dtype=np.float32)
    temp = np.empty((ids.size, N), dtype=np.float32) if with_temp else None
    jobs = [(spec, ids[lo:lo + chunk], with_temp) for lo in range(0, ids.size, chunk)]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for k, (r, v, t) in enumerate(ex.map(_skewers_chunk, jobs)):
            lo = k * chunk
            rho[lo:lo + r.shape[0]] = r
            vpec[lo:lo + r.shape[0]] = v
            if with_temp:
                temp[lo:lo + r.shape[0]] = t
    return rho, vpec, temp


# ---- rows of a large periodic grid --------------------------------------------------
# A 1536^3 grid has 2.36 million rows: drawing each one from its own seed on
# the host would take minutes and 43 GB of host memory.  Row r of such a grid
# is instead pool row (r mod P), cyclically shifted by ((r div P) * 997) mod N
# pixels.  A periodic shift of a periodic realisation is itself a valid
# realisation, so every row is a skewer with the stated statistics, distinct
# from every other row.
GRID_POOL_ROWS = 16384


def grid_row_shift(row_ids, n_pix: int, pool: int = GRID_POOL_ROWS) -> np.ndarray:
    row_ids = np.asarray(row_ids, dtype=np.int64)
    return ((row_ids // pool) * 997) % n_pix


def grid_rows(spec: FieldSpec, row_ids, pool: int = GRID_POOL_ROWS, with_temp: bool = True):
    """Host arrays of the given grid rows (same layout as :func:`skewers`)."""
    row_ids = np.asarray(row_ids, dtype=np.int64).ravel()
    base, shift = row_ids % pool, grid_row_shift(row_ids, spec.n_pix, pool)
    r, v, t = skewers(spec, base, with_temp=with_temp)
    out = []
    for a in (r, v, t):
        if a is None:
            out.append(None)
            continue
        b = np.empty_like(a)
        for k, s in enumerate(shift):
            b[k] = np.roll(a[k], int(s))
        out.append(b)
    return tuple(out)


def grid_on_device(spec: FieldSpec, n_rows: int, torch, device="cuda", pool: int = GRID_POOL_ROWS,
                   with_temp: bool = True, chunk: int = 8192):
    """Build all n_rows grid rows on the device (torch tensors [n_rows][N]).

    The pool is drawn on the host (parallel, seeded per row) and copied once;
    the rows are gathered from it on the device, chunk by chunk.
    """
    N = spec.n_pix
    pr, pv, pt = skewers_parallel(spec, np.arange(pool), with_temp=with_temp)
    pools = [torch.from_numpy(a).to(device) for a in (pr, pv, pt) if a is not None]
    outs = [torch.empty((n_rows, N), dtype=torch.float32, device=device) for _ in pools]
    cols = torch.arange(N, device=device)
    for lo in range(0, n_rows, chunk):
        rows = torch.arange(lo, min(lo + chunk, n_rows), device=device)
        base = rows % pool
        shift = ((rows // pool) * 997) % N
        idx = (cols[None, :] - shift[:, None]) % N          # out[i] = pool[(i - s) mod N]
        for src, dst in zip(pools, outs):
            dst[lo:lo + rows.numel()] = torch.gather(src[base], 1, idx)
    del pools
    return tuple(outs) + ((None,) if not with_temp else ())


# ---- a served request stream --------------------------------------------------------
# A pool of resident fields (density and velocity only; the temperature comes
# from each request's own power law): boxes log-uniform in [50, 1000] h^-1 Mpc,
# skewer lengths from {512, ..., 8192}, the paper-scale field recipe (k_J = 4,
# sigma_delta = 1.5, z = 2.5).  Requests arrive as a Poisson stream; each names
# a field of the pool, a log-uniform number of its skewers, its own T0, gamma
# and target mean flux.
SERVE_N_PIX = (512, 1024, 2048, 4096, 8192)
SERVE_BOX_RANGE = (50.0, 1000.0)
SERVE_SKEWERS_PER_FIELD = 4096
SERVE_RATE = 200.0                 # requests per second
SERVE_SEED = 3


@dataclass(frozen=True)
class ServeRequest:
    t_arrival: float               # seconds after the stream starts
    field: int                     # index into the pool
    ids: np.ndarray                # skewer ids of the field
    T0: float
    gamma: float
    target: float                  # mean flux the request is rescaled to


def serve_field_specs(boxes_per_length: int = 4, seed: int = SERVE_SEED) -> list:
    """The pool: ``boxes_per_length`` fields for every skewer length."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0]))
    lo, hi = np.log(SERVE_BOX_RANGE[0]), np.log(SERVE_BOX_RANGE[1])
    specs = []
    for n in SERVE_N_PIX:
        for b in range(boxes_per_length):
            box = float(np.exp(rng.uniform(lo, hi)))
            specs.append(FieldSpec(n_pix=n, box=box, z=2.5, k_j=4.0, sigma_delta=1.5, T0=1.5e4, gamma=1.5,
                                   seed=seed * 1000 + len(specs)))
    return specs


def serve_requests(n_fields: int, count: int, rate: float = SERVE_RATE, seed: int = SERVE_SEED,
                   skewers_per_field: int = SERVE_SKEWERS_PER_FIELD, max_skewers: int = 4096) -> list:
    """``count`` requests of a Poisson stream at ``rate`` per second."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
    t = 0.0
    out = []
    top = min(max_skewers, skewers_per_field)
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        f = int(rng.integers(n_fields))
        n = int(np.clip(np.round(np.exp(rng.uniform(0.0, np.log(top)))), 1, top))
        ids = np.sort(rng.choice(skewers_per_field, size=n, replace=False)).astype(np.int64)
        out.append(ServeRequest(t, f, ids, float(rng.uniform(1.0e4, 2.5e4)), float(rng.uniform(1.0, 1.6)),
                                float(rng.uniform(0.65, 0.85))))
    return out
