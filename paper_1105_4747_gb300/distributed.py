"""Mean-flux root-find over pixels split across devices or processes (Sec. 2.3).

A request's optical depths may live on several GPUs (a skewer set sharded by
rank).  A is one number for all of them.  The library does all of the
method's arithmetic: each part's shares of the sums (lya_tau_moments,
lya_mean_flux_sums) and the iteration itself (lya_mean_flux_start /
lya_mean_flux_step, or the whole loop in lya_rescale_mean_flux_sharded).
This module only supplies the all-reduce that sums the shares over the
parts (three or four FP64 numbers per pass) and maps the library's errors to
exceptions.
"""
from __future__ import annotations

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


def _raise(exc, target):
    from ._binding import LYA_EINVAL, LYA_ENOCONV
    if exc.status == LYA_ENOCONV:
        raise NoConvergence(f"mean-flux root-find: no convergence to <F> = {target} ({exc})") from exc
    if exc.status == LYA_EINVAL:
        raise ValueError(f"mean-flux root-find: {exc}") from exc
    raise exc


def rescale_mean_flux_distributed(tau, target: float, *, n: int | None = None,
                                  allreduce: Callable[[Sequence[float]], Sequence[float]] | None = None,
                                  moments: Callable[[], Sequence[float]] | None = None,
                                  sums: Callable[[float], Sequence[float]] | None = None,
                                  tol: float = 1e-12, max_iter: int = 50) -> tuple[float, int]:
    """A with <exp(-A tau)> = target over the union of every part's ``tau``.

    ``allreduce`` sums a list of floats over all parts (default:
    torch.distributed, SUM).  With neither ``moments`` nor ``sums`` the
    library runs the whole split root-find on this part's device tensor
    ``tau`` (lya_rescale_mean_flux_sharded).  Otherwise ``moments()`` gives
    this part's (sum tau, zeros, invalid) and ``sums(A)`` its (sum e, sum tau
    e, sum tau^2 e), and the library steps the iteration on their all-reduced
    totals (``n``: this part's number of values).  Returns ``(A, passes)``.
    """
    if not (0.0 < target < 1.0):
        raise ValueError("target mean flux must be in (0, 1)")
    from ._binding import LyaError, mean_flux_start, mean_flux_step, rescale_mean_flux_sharded
    if allreduce is None:
        allreduce = _torch_allreduce
    try:
        if moments is None and sums is None:
            A, steps, _ = rescale_mean_flux_sharded(tau, target, allreduce, tol=tol, max_iter=max_iter,
                                                    flux_out=None)
            return A, steps
        if moments is None or sums is None:
            from ._binding import mean_flux_sums, tau_moments
            moments = moments or (lambda: tau_moments(tau))
            sums = sums or (lambda A: mean_flux_sums(tau, A))
        local_n = float(tau.numel() if n is None else n)
        it = mean_flux_start(allreduce(list(moments()) + [local_n]), target, tol=tol, max_iter=max_iter)
        while not it.done:
            mean_flux_step(it, allreduce(list(sums(it.A))))
        return it.A, it.iter
    except LyaError as exc:
        _raise(exc, target)
