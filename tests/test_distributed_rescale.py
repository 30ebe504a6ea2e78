"""The mean-flux root-find over pixels split across processes (gloo, CPU).

Two ranks each hold half of the optical depths; their shares of the sums are
combined with torch.distributed all-reduce (gloo on 127.0.0.1) and both step
the iteration with the library's C calls (lya_mean_flux_start /
lya_mean_flux_step, host code: no GPU needed).  The per-part sums here are
plain FP64 numpy (the stand-in for the library's per-device share on a
CPU-only machine); the result must equal the oracle's A over all pixels, and
the steps must be the library's (the Python layer does no arithmetic of the
method)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, tau_all, target, out_path):
    import torch.distributed as dist
    from paper_1105_4747_gb300.distributed import NoConvergence, rescale_mean_flux_distributed
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    part = np.array_split(tau_all, world)[rank].astype(np.float64)

    def moments():
        return [part.sum(), float((part == 0).sum()), float((~np.isfinite(part) | (part < 0)).sum())]

    def sums(A):
        e = np.exp(-A * part)
        return [e.sum(), (part * e).sum(), (part * part * e).sum()]

    try:
        A, it = rescale_mean_flux_distributed(None, target, n=part.size, moments=moments, sums=sums)
        res = f"{A!r} {it}"
    except NoConvergence:
        res = "noconv"
    np.save(f"{out_path}.{rank}.npy", np.array([res]))
    dist.barrier()
    dist.destroy_process_group()


def _run(tau_all, target, tmp_path, world=2):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res")
    mp.start_processes(_rank_main, args=(world, _free_port(), tau_all, target, out), nprocs=world,
                       start_method="spawn", join=True)
    return [str(np.load(f"{out}.{r}.npy")[0]) for r in range(world)]


def test_two_ranks_match_the_oracle(tmp_path):
    import oracle
    import lya_synth as ls
    oracle.build()
    spec = ls.TINY_20MPC
    rho, v, t = ls.skewers(spec, np.arange(16))
    tau = oracle.tau(oracle.Params(box=spec.box, z=spec.z), rho, v, t).astype(np.float32).ravel()
    res = _run(tau, 0.8, tmp_path)
    A0, it0 = res[0].split()
    A1, it1 = res[1].split()
    assert A0 == A1 and it0 == it1              # both ranks take the same steps
    A_ref, _ = oracle.rescale(tau.astype(np.float64), 0.8)
    assert float(A0) == pytest.approx(A_ref, rel=1e-11)


def test_host_steps_match_the_oracle_in_one_process():
    """lya_mean_flux_start / lya_mean_flux_step driven directly with FP64
    sums: the library's steps reach the oracle's A, and the certified stop
    leaves |<exp(-A tau)> - F_t| within 1e-12."""
    import oracle
    import lya_synth as ls
    from paper_1105_4747_gb300 import _binding as b
    oracle.build()
    spec = ls.TINY_20MPC
    rho, v, t = ls.skewers(spec, np.arange(8))
    tau = oracle.tau(oracle.Params(box=spec.box, z=spec.z), rho, v, t).astype(np.float32).astype(np.float64).ravel()
    for target in (0.8, 0.6, 0.95):
        it = b.mean_flux_start([tau.sum(), float((tau == 0).sum()), 0.0, float(tau.size)], target)
        while not it.done:
            e = np.exp(-it.A * tau)
            b.mean_flux_step(it, [e.sum(), (tau * e).sum(), (tau * tau * e).sum()])
        assert it.status == 0
        A_ref, _ = oracle.rescale(tau, target)
        assert it.A == pytest.approx(A_ref, rel=1e-11)
        assert abs(float(np.mean(np.exp(-it.A * tau))) - target) <= 1e-12
    with pytest.raises(b.LyaError):
        b.mean_flux_start([10.0, 90.0, 0.0, 100.0], 0.85)          # 90 % of tau = 0: no root


def test_two_ranks_agree_on_no_root(tmp_path):
    tau = np.array([0.0] * 90 + [1.0] * 10, dtype=np.float32)
    assert _run(tau, 0.85, tmp_path) == ["noconv", "noconv"]
