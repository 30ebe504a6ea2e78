"""Mean-flux root-find over pixels split across devices or processes (Sec. 2.3).

A request's optical depths may live on several GPUs (a skewer set sharded by
rank).  A is one number for all of them: each part computes its share of the
sums with the library (lya_tau_moments, lya_mean_flux_sums), the shares are
summed with one all-reduce of three FP64 numbers per pass, and every part
takes the same safeguarded Halley step that the single-device kernel takes:
Newton on g(A) = <exp(-A tau)> - F_t from the Jensen bound
A0 = -ln(F_t)/<tau>, Halley's step when it stays inside the bracket, else
Newton's, else bisection; stop at |g| <= tol or when the step stalls at FP64
resolution.  Only these three scalars cross the host; all per-pixel work is
in the library's kernels.
"""
from __future__ import annotations

import math
from typing import Callable, Sequence


class NoConvergence(RuntimeError):
    pass


def _torch_allreduce(values: Sequence[float]):
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()]


def rescale_mean_flux_distributed(tau, target: float, *, n: int | None = None,
                                  allreduce: Callable[[Sequence[float]], Sequence[float]] | None = None,
                                  moments: Callable[[], Sequence[float]] | None = None,
                                  sums: Callable[[float], Sequence[float]] | None = None,
                                  tol: float = 1e-12, max_iter: int = 50) -> tuple[float, int]:
    """A with <exp(-A tau)> = target over the union of every part's ``tau``.

    ``allreduce`` sums a list of floats over all parts (default: torch.distributed,
    SUM); ``moments``/``sums`` give this part's shares (default: the library on
    this part's device tensor ``tau``).  Returns ``(A, passes)``.
    """
    if not (0.0 < target < 1.0):
        raise ValueError("target mean flux must be in (0, 1)")
    if allreduce is None:
        allreduce = _torch_allreduce
    if moments is None or sums is None:
        from ._binding import mean_flux_sums, tau_moments
        moments = moments or (lambda: tau_moments(tau))
        sums = sums or (lambda A: mean_flux_sums(tau, A))
    local_n = float(tau.numel() if n is None else n)
    s_tau, n_zero, n_bad, n_tot = allreduce(list(moments()) + [local_n])
    if n_bad > 0 or not (s_tau > 0.0):
        raise ValueError("tau holds a negative or non-finite value, or is all zero")
    if n_zero / n_tot >= target:
        raise NoConvergence(f"no A reaches <F> = {target}: {n_zero / n_tot:.3g} of the pixels have tau = 0")
    A = -math.log(target) / (s_tau / n_tot)
    lo, hi = A, math.inf
    for it in range(1, max_iter + 1):
        s0, s1, s2 = allreduce(sums(A))
        g = s0 / n_tot - target
        g1, g2 = -s1 / n_tot, s2 / n_tot
        if abs(g) <= tol:
            return A, it
        if g > 0:
            lo = A
        else:
            hi = A
        den = 2.0 * g1 * g1 - g * g2
        An = A - 2.0 * g * g1 / den if den > 0 else math.nan
        if not (lo < An < hi):
            An = A - g / g1 if g1 < 0 else math.nan
        if not (lo < An < hi):
            An = 0.5 * (lo + hi) if math.isfinite(hi) else 2.0 * lo
        if abs(An - A) <= 4e-16 * abs(A):
            return A, it
        A = An
    raise NoConvergence(f"mean-flux root-find did not converge in {max_iter} passes")
