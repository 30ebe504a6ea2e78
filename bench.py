#!/usr/bin/env python
"""Benchmark of the Lyman-alpha optical-depth hot path on GB300.

One step = one pass of the whole path over the 65,536 x 4,096-pixel skewer
field of a periodic 1 h^-1 Gpc box at z = 2.5 (stored temperature,
gamma = 1.5, target <F> = 0.80): optical depth of every skewer (Eq. 4-6),
the mean-flux root-find and F = exp(-A tau) (Sec. 2.3), and the flux
statistics (Sec. 5.2).  The metric is output pixels per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``value`` is timed with CUDA events on the launching stream with the inputs
resident in HBM (3.2 GB of inputs, far above the 129 MB L2, so no flush is
needed between steps); ``e2e`` repeats the step through the public API with
the inputs copied from pinned host memory and F copied back every step.
Under torchrun each rank runs an independent replica of the workload (weak
scaling); rank 0 prints one JSON line with the max-over-ranks time.
``--impl reference`` times the FP64 CPU oracle on the host cores on bounded
samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lya_synth as ls  # noqa: E402

METRIC = "tau-skewer pixels/s on 1 GB300 at |dF|<=1e-5 vs FP64 oracle"
UNIT = "pixels/s"
WORKLOAD = "gpc_box_65536x4096_z2.5"
ALG_BYTES_PER_PX = 16          # rho, vpec, T read (12 B) + tau written (4 B)
# DRAM bytes of one tau-kernel launch per skewer, from the ncu captures in
# profiles/ (8,192 skewers of the Gpc workload; 131,072 rows of the grid),
# scaled by the number of skewers, with the SHA-1 of the kernel source each
# was taken on: reported as null once paper_1105_4747_gb300/csrc/tau_extract.cu
# differs from it.
TAU_DRAM_PROFILE = {"gpc": ((402.798592e6 + 113.191424e6) / 8192, "c274fd95e764757eb255cf1ac4ecf05cf9974d4f"),
                    "grid1536": ((2.416186112e9 + 0.75963264e9) / 131072, "c274fd95e764757eb255cf1ac4ecf05cf9974d4f")}


# ncu pipe utilisation of the same tau-kernel launch as TAU_DRAM_PROFILE["gpc"]
# (8,192 skewers, --set full, profiles/tau_tile_kernel_gpc_8192x4096.md), with
# the code hash it was taken on: reported as null once the kernel differs.
TAU_PIPE_PROFILE = {"gpc": ({"fma_pct": 19.4, "xu_pct": 20.4, "alu_pct": 46.1, "lsu_pct": 19.3,
                             "issue_active_pct": 67.5}, "c274fd95e764757eb255cf1ac4ecf05cf9974d4f")}
FP32_OPS_PER_PAIR = 6          # per pair of the sum: argument (2), square, exponent scale, weight, add
KB_J_PER_K = 1.380649e-23
M_H_KG = 1.6735575e-27


def algorithmic_pairs_per_px(rho, v, t, du, window=8.0):
    """Pairs (i, j) of the Eq. 6 sum within the window: |i du - (j du + v_j)| <= window b_j,
    b_j = (2 k T_j / m_H)^(1/2), counted exactly on host rows (sources with rho > 0),
    per output pixel."""
    rho = np.asarray(rho, dtype=np.float64)
    N = rho.shape[1]
    u = np.arange(N)[None, :] * du + np.asarray(v, dtype=np.float64)
    b = np.sqrt(2.0 * KB_J_PER_K * np.asarray(t, dtype=np.float64) / M_H_KG) / 1e3
    lo = np.ceil((u - window * b) / du)
    hi = np.floor((u + window * b) / du)
    cnt = np.clip(hi - lo + 1.0, 0.0, float(N))
    return float(cnt[rho > 0].sum() / rho.size)


def tau_code_hash() -> str:
    """SHA-1 of the optical-depth kernel's code: tau_extract.cu and the headers
    it includes, with comments and blank lines removed (a comment edit does not
    change the kernel whose DRAM traffic was captured)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1105_4747_gb300", "csrc")
    h = hashlib.sha1()
    for name in ("tau_extract.cu", "lya_device.cuh", "lya_internal.h", "serve_internal.h"):
        txt = open(os.path.join(csrc, name)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        h.update("\n".join(line.rstrip() for line in txt.splitlines() if line.strip()).encode())
    return h.hexdigest()


def workload_config(spec, S, extra=None, grid=False):
    c = {"workload": "grid_1536cubed_z2.3" if grid else WORKLOAD, "n_skewers": S, "n_pix": spec.n_pix,
         "box_mpc_h": spec.box, "z": spec.z, "T": "stored", "gamma": spec.gamma,
         "target_mean_flux": ls.GRID_1536_FT if grid else ls.GPC_4096_FT,
         "precision": "f32 pairs, compensated sum; f64 root-find",
         "l2": ("inputs 43.5 GB" if grid else "inputs 3.2 GB") + " > 129 MB L2: no flush between steps"}
    if extra:
        c.update(extra)
    return c


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample_run(spec, ids, rho, v, t):
    import oracle
    p = oracle.Params(box=spec.box, z=spec.z, t_mode=0)
    t0 = time.perf_counter()
    tau = oracle.tau(p, rho, v, t)
    A, _ = oracle.rescale(tau, ls.GPC_4096_FT)
    F = oracle.flux(tau, A)
    oracle.flux_stats(F)
    return time.perf_counter() - t0


def oracle_timing(spec, seconds: float, seed: int = 7):
    """Time the oracle on a sample sized to take about `seconds`."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    rng = np.random.default_rng(seed)
    n = cores
    ids = np.sort(rng.choice(ls.GPC_4096_SKEWERS, n, replace=False))
    r, v, t = ls.skewers(spec, ids)
    dt = oracle_sample_run(spec, ids, r, v, t)
    n2 = int(max(cores, min(4096, round(seconds / max(dt, 1e-3) * n / cores) * cores)))
    ids = np.sort(rng.choice(ls.GPC_4096_SKEWERS, n2, replace=False))
    r, v, t = ls.skewers(spec, ids)
    dt = oracle_sample_run(spec, ids, r, v, t)
    px = n2 * spec.n_pix
    return {"value": px / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n2} random skewers x {spec.n_pix} px of the workload (full O(N^2) FP64 sum, "
                      f"rescale to <F>=0.80, stats) in {dt:.1f} s"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    spec = ls.GPC_4096
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    rng = np.random.default_rng(1234)
    per_step = max(cores, 2 * cores)
    times, px = [], 0
    for step in range(args.warmup + args.steps):
        ids = np.sort(rng.choice(ls.GPC_4096_SKEWERS, per_step, replace=False))
        r, v, t = ls.skewers(spec, ids)
        dt = oracle_sample_run(spec, ids, r, v, t)
        if step >= args.warmup:
            times.append(dt)
            px += per_step * spec.n_pix
    total = sum(times)
    value = px / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(spec, ls.GPC_4096_SKEWERS,
                                                           {"sample_per_step": f"{per_step} skewers"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random skewers x {spec.n_pix} px per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the served form: Poisson arrivals into the library's serving loop
# ---------------------------------------------------------------------------
SERVE_BUDGET = 120 << 30                 # HBM budget of admitted requests (tau + F)


def serving_pool(lya, torch, boxes_per_length=4, pool_rows=256):
    """The resident field pool (density and velocity), built on the device."""
    specs = ls.serve_field_specs(boxes_per_length)
    fields = []
    for sp in specs:
        rho, v, _ = ls.grid_on_device(sp, ls.SERVE_SKEWERS_PER_FIELD, torch, pool=pool_rows, with_temp=False)
        fields.append(lya.Field(rho, v, None, box=sp.box, z=sp.z, borrow=True))
    return specs, fields


def serve_stream(lya, srv, fields, reqs, t_end):
    """Submit ``reqs`` at their arrival times (until t_end s) from one thread,
    wait for and release each from another; returns [(request, result)], the
    submitter's lateness (s) per request and the stream's start (ns)."""
    import queue
    q = queue.Queue()
    done, lag = [], []
    t0 = time.monotonic() + 0.05

    def submitter():
        for r in reqs:
            if r.t_arrival > t_end:
                break
            dt = t0 + r.t_arrival - time.monotonic()
            if dt > 0:
                time.sleep(dt)
            lag.append(time.monotonic() - (t0 + r.t_arrival))
            tk = srv.submit(fields[r.field], lya.ExtractParams(t_mode=1, T0=r.T0, gamma=r.gamma), r.ids, r.target)
            q.put((r, tk))
        q.put(None)

    def reaper():
        while True:
            item = q.get()
            if item is None:
                return
            r, tk = item
            res = srv.wait(tk, 600.0)
            done.append((r, res))
            srv.release(tk)

    th = [threading.Thread(target=submitter), threading.Thread(target=reaper)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return done, lag, int(t0 * 1e9)


# bytes per served pixel the step moves: Delta and v read (8), tau written and
# read back by the init and two Halley passes (4 + 12), F written by the flux
# pass after reading tau (8)
SERVE_BYTES_PER_PX = 32


def serving_pairs_per_px(specs, rows=16, T0=1.75e4, gamma=1.3, pivot=10.0):
    """Algorithmic pairs per pixel of the served stream: every pool field's
    pairs per pixel on a few host rows with the middle of the requests'
    temperature range (T = T0 min(1 + delta, pivot)^(gamma - 1)), weighted
    by skewer length (requests pick fields uniformly, so pixels go as n_pix)."""
    num = den = 0.0
    for sp in specs:
        r, v, _ = ls.grid_rows(sp, np.arange(rows), with_temp=False)
        T = T0 * np.minimum(r.astype(np.float64), pivot) ** (gamma - 1.0)
        e = np.sqrt(sp.omega_m * (1 + sp.z) ** 3 + sp.omega_l)
        du = 100.0 * e / (1 + sp.z) * sp.box / sp.n_pix
        num += algorithmic_pairs_per_px(r, v, T, du) * sp.n_pix
        den += sp.n_pix
    return num / den


def run_serving(lya, torch, warm_s, measure_s, burst=400, budget=SERVE_BUDGET, peaks=None, sms=152, clk_hz=2.07e9):
    """p50/p99 latency and served pixels/s of the Poisson stream, and the
    loop's capacity (a burst of requests submitted at once) with its
    rooflines."""
    specs, fields = serving_pool(lya, torch)
    reqs = ls.serve_requests(len(fields), int((warm_s + measure_s) * ls.SERVE_RATE * 1.5) + burst)
    srv = lya.Server(budget_bytes=budget, max_slots=256, step_target_us=2000.0)
    shifts = {}
    for n in ls.SERVE_N_PIX:
        k = [i for i, sp in enumerate(specs) if sp.n_pix == n]
        mid = sorted(k, key=lambda i: specs[i].box)[len(k) // 2]
        shifts[n] = srv.autotune(fields[mid], lya.ExtractParams(t_mode=1, T0=1.75e4, gamma=1.3), max_rows=1024)
    info0 = srv.info()
    launches0 = lya.kernel_launches()
    done, lag, t0_ns = serve_stream(lya, srv, fields, reqs, warm_s + measure_s)
    launches = lya.kernel_launches() - launches0
    info1 = srv.info()
    w0, w1 = t0_ns + int(warm_s * 1e9), t0_ns + int((warm_s + measure_s) * 1e9)
    lat, px_done, px_offered, n_meas, failed = [], 0, 0, 0, 0
    for r, res in done:
        px = r.ids.size * specs[r.field].n_pix
        if res.status != 0:
            failed += 1
        if warm_s <= r.t_arrival < warm_s + measure_s:
            lat.append((res.t_done_ns - res.t_submit_ns) * 1e-6)
            px_offered += px
            n_meas += 1
        if w0 <= res.t_done_ns < w1:
            px_done += px
    lat = np.array(lat)
    # capacity: a burst of the next requests, all submitted at once
    tail = reqs[len(done):len(done) + burst]
    t_b0 = time.monotonic_ns()
    tickets = [srv.submit(fields[r.field], lya.ExtractParams(t_mode=1, T0=r.T0, gamma=r.gamma), r.ids, r.target)
               for r in tail]
    last, px_b = 0, 0
    for r, tk in zip(tail, tickets):
        res = srv.wait(tk, 600.0)
        last = max(last, res.t_done_ns)
        px_b += r.ids.size * specs[r.field].n_pix
        srv.release(tk)
    cap = px_b / ((last - t_b0) * 1e-9)
    srv.close()
    for f in fields:
        f.close()
    pairs_px = serving_pairs_per_px(specs)
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    roofline = {"fp32_pipe": fp32_pipe(pairs_px, 1.0, 1e3 / cap, sms, clk_hz), "alg_pairs_per_px": pairs_px,
                "hbm": {"achieved": cap * SERVE_BYTES_PER_PX / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": cap * SERVE_BYTES_PER_PX / 1e9 / hbm, "bytes_per_px": SERVE_BYTES_PER_PX},
                "at": "capacity (the burst), whole served step: extraction, root-find and statistics"}
    return {"workload": f"poisson_{ls.SERVE_RATE:g}rps_pool{len(fields)}x{ls.SERVE_SKEWERS_PER_FIELD}",
            "rate_rps": ls.SERVE_RATE, "warmup_s": warm_s, "measure_s": measure_s, "requests": n_meas,
            "failed": failed, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "served_px_per_s": px_done / measure_s, "offered_px_per_s": px_offered / measure_s,
            "capacity_px_per_s": cap, "capacity_burst_requests": len(tail), "roofline": roofline,
            "p99_samples": int(len(lat)), "p99_tail_samples": int(round(0.01 * len(lat))),
            "submit_lag_p99_ms": float(np.percentile(np.array(lag), 99) * 1e3),
            "steps": info1["steps"] - info0["steps"], "gpu_launches": launches,
            "group_shift_by_n_pix": {str(k): v for k, v in shifts.items()},
            "budget_bytes": budget, "latency": "submit to result (native steady clock)",
            "data": "synthetic pool: boxes log-uniform 50-1000 h^-1 Mpc, n_pix 512-8192, T from each request's "
                    "power law"}


def run_post(lya, torch, field, F, S, spec, reps):
    """Timings of lya_mock_spectra (the BOSS-like instrument of Sec. 4) and
    lya_flux_power_1d on the step's F, with their HBM rooflines."""
    c_kms = 2.99792458e5
    du = lya.field_pixel_width(field)
    p = lya.MockParams(fwhm_kms=224.0, bin_kms=c_kms * 1.0375 / (1215.67 * (1.0 + spec.z)), snr=5.0,
                       max_kms=c_kms * np.log(1215.67 / 1025.72) - 3000.0, seed=11)
    out = lya.mock_spectra(F, du, p)
    M = out.shape[1]
    lya.flux_power_1d(F, du)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    for _ in range(reps):
        lya.mock_spectra(F, du, p, out=out)
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(reps):
        lya.flux_power_1d(F, du)
    ev[3].record(stream)
    ev[3].synchronize()
    ms_mock = ev[0].elapsed_time(ev[1]) / reps
    ms_ps = ev[2].elapsed_time(ev[3]) / reps
    # Fourier-space generation of the same number of lines of sight (Sec. 2.1-2.2)
    gkw = dict(box=spec.box, z=spec.z, k_j=spec.k_j, sigma_delta=spec.sigma_delta, seed=spec.seed)
    g_rho = torch.empty((S, spec.n_pix), dtype=torch.float32, device="cuda")
    g_v = torch.empty_like(g_rho)
    lya.generate_sightlines(spec.n_pix, 0, S, rho_out=g_rho, vpec_out=g_v, **gkw)
    ev[0].record(stream)
    for _ in range(reps):
        lya.generate_sightlines(spec.n_pix, 0, S, rho_out=g_rho, vpec_out=g_v, **gkw)
    ev[1].record(stream)
    ev[1].synchronize()
    ms_gen = ev[0].elapsed_time(ev[1]) / reps
    del g_rho, g_v
    # the Eq. 7 3D flux power of a 64 x 64 grid of lines (4,096 of the step's
    # skewers): the density of a 45 deg^-2 survey across a 1 h^-1 Gpc box
    n_perp = 64
    Fs = F[: n_perp * n_perp]
    cells = np.arange(n_perp * n_perp)
    lya.flux_power_3d(Fs, cells, n_perp, spec.box)
    ev[0].record(stream)
    for _ in range(reps):
        lya.flux_power_3d(Fs, cells, n_perp, spec.box)
    ev[1].record(stream)
    ev[1].synchronize()
    ms_3d = ev[0].elapsed_time(ev[1]) / reps
    b_3d = 2 * 4 * n_perp * n_perp * spec.n_pix + 2 * 8 * (spec.n_pix // 2 + 1) * n_perp * n_perp
    # the pixel-averaged line profile (column-conserving variant of Eq. 6)
    p_avg = lya.ExtractParams(t_mode=0, profile=lya.PROFILE_AVERAGED)
    tau_avg = torch.empty((S, spec.n_pix), dtype=torch.float32, device="cuda")
    lya.extract_skewers(field, p_avg, out=tau_avg)
    ev[0].record(stream)
    for _ in range(reps):
        lya.extract_skewers(field, p_avg, out=tau_avg)
    ev[1].record(stream)
    ev[1].synchronize()
    ms_avg = ev[0].elapsed_time(ev[1]) / reps
    del tau_avg
    # an oversampled field (b/du ~ 26: 8,192-pixel lines of sight through a
    # 50 h^-1 Mpc box, the short end of the served boxes), generated on the
    # device, extracted with each way of forming the pair sum's exponentials
    o_n, o_S, o_box = 8192, 4096, 50.0
    o_rho = torch.empty((o_S, o_n), dtype=torch.float32, device="cuda")
    o_v = torch.empty_like(o_rho)
    lya.generate_sightlines(o_n, 0, o_S, rho_out=o_rho, vpec_out=o_v, box=o_box, z=spec.z, k_j=spec.k_j,
                            sigma_delta=spec.sigma_delta, seed=spec.seed + 1)
    o_field = lya.Field(o_rho, o_v, None, box=o_box, z=spec.z, borrow=True)
    o_tau = torch.empty_like(o_rho)
    o_ms = {}
    for name, em in (("mufu", lya.EXP_MUFU), ("recurrence", lya.EXP_RECURRENCE),
                     ("poly_split", lya.EXP_POLY_SPLIT)):
        p_o = lya.ExtractParams(t_mode=1, T0=1.5e4, gamma=1.5, exp_method=em)
        lya.extract_skewers(o_field, p_o, out=o_tau)
        ev[0].record(stream)
        for _ in range(reps):
            lya.extract_skewers(o_field, p_o, out=o_tau)
        ev[1].record(stream)
        ev[1].synchronize()
        o_ms[name] = ev[0].elapsed_time(ev[1]) / reps
    o_du = lya.field_pixel_width(o_field)
    o_field.close()
    del o_rho, o_v, o_tau
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    n_px = S * spec.n_pix
    b_mock = 4 * n_px + 4 * S * M            # read F, write the mock pixels
    b_ps = 8 * n_px                          # F read by the mean pass and by the transform pass
    return {"mock_spectra": {"instrument": "FWHM 224 km/s, 1.0375 A pixels, S/N 5, Ly-alpha to Ly-beta path less "
                                           "3000 km/s (Sec. 4)", "n_out_pix": M, "ms": ms_mock,
                             "input_px_per_s": n_px / (ms_mock / 1e3),
                             "roofline": {"bound": "hbm", "achieved": b_mock / (ms_mock / 1e3) / 1e9, "peak": peak,
                                          "unit": "GB/s", "frac": b_mock / (ms_mock / 1e3) / 1e9 / peak,
                                          "alg_bytes_per_launch": b_mock}},
            "tau_oversampled": {"workload": f"{o_S} lines x {o_n} px, {o_box:g} h^-1 Mpc box (du {o_du:.3f} km/s, "
                                            "T = 1.5e4 K Delta^0.5), generated on the device",
                                "ms": o_ms, "px_per_s": {k: o_S * o_n / (v / 1e3) for k, v in o_ms.items()},
                                "note": "tau_tile_kernel, 1,024-thread CTAs, four-pixel lanes; exp_method mufu "
                                        "(one MUFU ex2 per pair), recurrence (Gaussian recurrence, three MUFU per "
                                        "four pairs), poly_split (one exp2 in four on the FMA pipe)"},
            "tau_averaged_profile": {"ms": ms_avg, "px_per_s": n_px / (ms_avg / 1e3),
                                     "roofline": {"bound": "hbm", "achieved": 16 * n_px / (ms_avg / 1e3) / 1e9,
                                                  "peak": peak, "unit": "GB/s",
                                                  "frac": 16 * n_px / (ms_avg / 1e3) / 1e9 / peak,
                                                  "alg_bytes_per_launch": 16 * n_px},
                                     "note": "tau_tile_kernel with four erfc per candidate and lane"},
            "flux_power_3d": {"ms": ms_3d, "lines": n_perp * n_perp, "n_perp": n_perp,
                              "roofline": {"bound": "hbm", "achieved": b_3d / (ms_3d / 1e3) / 1e9, "peak": peak,
                                           "unit": "GB/s", "frac": b_3d / (ms_3d / 1e3) / 1e9 / peak,
                                           "alg_bytes_per_launch": b_3d},
                              "note": "F read twice, the k_z planes written and read; host round trip included"},
            "sightlines": {"ms": ms_gen, "px_per_s": n_px / (ms_gen / 1e3),
                           "roofline": {"bound": "hbm", "achieved": 8 * n_px / (ms_gen / 1e3) / 1e9, "peak": peak,
                                        "unit": "GB/s", "frac": 8 * n_px / (ms_gen / 1e3) / 1e9 / peak,
                                        "alg_bytes_per_launch": 8 * n_px},
                           "note": "1 + delta and v_pec written (8 B/px), modes drawn on the device"},
            "flux_power_1d": {"ms": ms_ps, "input_px_per_s": n_px / (ms_ps / 1e3),
                              "roofline": {"bound": "hbm", "achieved": b_ps / (ms_ps / 1e3) / 1e9, "peak": peak,
                                           "unit": "GB/s", "frac": b_ps / (ms_ps / 1e3) / 1e9 / peak,
                                           "alg_bytes_per_launch": b_ps},
                              "note": "includes the host round trip of the call (it synchronises)"}}


def run_e2e(lya, torch, field, spec, S, params, target, rho, v, t, tau, F, n_steps, world, local):
    """Pipelined end-to-end steps through the public API (see run_ours)."""
    n_px = S * spec.n_pix
    rho_h = torch.from_numpy(rho).pin_memory()
    v_h = torch.from_numpy(v).pin_memory()
    t_h = torch.from_numpy(t).pin_memory()
    F_h = [torch.empty((S, spec.n_pix), dtype=torch.float32).pin_memory() for _ in range(2)]
    fields = [field, lya.Field(rho_h, v_h, t_h, box=spec.box, z=spec.z)]
    Fd = [F, torch.empty_like(F)]
    s_load, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    comp = torch.cuda.current_stream()
    ready = [threading.Event() for _ in range(n_steps)]
    free = [threading.Semaphore(1), threading.Semaphore(1)]
    out_ev = [None, None]
    errors = []

    def loader():
        try:
            torch.cuda.set_device(local)
            for k in range(n_steps):
                free[k % 2].acquire()
                fields[k % 2].load(rho_h, v_h, t_h, stream=s_load)     # returns when the copy landed
                ready[k].set()
        except Exception as exc:                                       # surfaced by the main thread
            errors.append(exc)
            for e in ready:
                e.set()

    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th = threading.Thread(target=loader)
    th.start()
    for k in range(n_steps):
        ready[k].wait()
        if errors:
            raise errors[0]
        b = k % 2
        if out_ev[b] is not None:
            out_ev[b].synchronize()                     # F[b] of step k-2 has reached the host
        lya.extract_skewers(fields[b], params, out=tau)
        lya.rescale_mean_flux_stats(tau, target, flux_out=Fd[b])   # returns when A and F are final
        free[b].release()                               # the loader may refill fields[b]
        with torch.cuda.stream(s_out):
            s_out.wait_stream(comp)
            F_h[b].copy_(Fd[b], non_blocking=True)
            out_ev[b] = torch.cuda.Event()
            out_ev[b].record(s_out)
    th.join()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dt, world)
    # the one-way bandwidth of these very host buffers (best of three 1-array
    # copies), beside the link measured on separate buffers: tells a slow
    # placement of the step's buffers apart from a slow pipeline
    dst = torch.empty(rho_h.shape, dtype=torch.float32, device="cuda")
    best = 0.0
    for _ in range(3):
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        dst.copy_(rho_h, non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, rho_h.numel() * 4 / (time.perf_counter() - c0) / 1e9)
    del dst
    fields[1].close()
    return {"value": world * n_steps * n_px / dt, "unit": UNIT,
            "h2d_bytes_per_step": 3 * n_px * 4, "d2h_bytes_per_step": n_px * 4,
            "ms_per_step": 1e3 * dt / n_steps, "steps": n_steps, "buffers_h2d_gbs": best,
            "timing": "host wall clock around all steps, device synchronised at both ends",
            "pipeline": "two device fields and two F buffers: H2D of step k+1 and D2H of step k-1 overlap step k"}


def fp64_mean_flux(torch, tau, A):
    """<exp(-A tau)> over every value of a device tensor in FP64 (torch, on the
    device, chunk by chunk): the defining property of A, reported beside it."""
    flat = tau.reshape(-1)
    total = torch.zeros((), dtype=torch.float64, device=flat.device)
    for lo in range(0, flat.numel(), 1 << 27):
        total += torch.exp(-A * flat[lo:lo + (1 << 27)].double()).sum()
    return float(total) / flat.numel()


def measure_link(torch, nbytes=1 << 30, reps=5):
    """Pinned host <-> device copy bandwidth (GB/s, best of reps, CUDA events):
    one way each, and both ways at once on two streams."""
    n = nbytes // 4
    h_in = torch.empty(n, dtype=torch.float32).pin_memory()
    h_out = torch.empty(n, dtype=torch.float32).pin_memory()
    d_in = torch.empty(n, dtype=torch.float32, device="cuda")
    d_out = torch.empty(n, dtype=torch.float32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best

    def both():
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)

    h2d = nbytes / timed(lambda: d_in.copy_(h_in, non_blocking=True)) / 1e9
    d2h = nbytes / timed(lambda: h_out.copy_(d_out, non_blocking=True)) / 1e9
    bi = 2 * nbytes / timed(both) / 1e9
    del h_in, h_out, d_in, d_out
    return {"h2d_gbs": h2d, "d2h_gbs": d2h, "both_ways_gbs": bi, "bytes_per_copy": nbytes,
            "how": "pinned host memory, 1 GiB copies, best of 5, host clock around synchronised copies"}


def fp32_pipe(pairs_px, n_px, ms, sms, clk_hz):
    """Algorithmic pair arithmetic of an extraction against the FP32 pipe peak."""
    peak = sms * 128 * clk_hz
    achieved = pairs_px * n_px * FP32_OPS_PER_PAIR / (ms / 1e3)
    return {"achieved": achieved, "peak": peak, "unit": "FP32 operations/s", "frac": achieved / peak}


def time_extract(lya, torch, field, params, out, reps):
    """Mean duration (ms, CUDA events) of extract_skewers over reps launches."""
    lya.extract_skewers(field, params, out=out)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        lya.extract_skewers(field, params, out=out)
    ev[1].record()
    ev[1].synchronize()
    return ev[0].elapsed_time(ev[1]) / reps


def run_precision_variants(lya, torch, field, spec, S, tau_ms_comp, pairs_px, sms, clk_hz, reps):
    """The optical depth of the same field with FP32 naive sums and with the
    FP64 comparator kernel, beside the FP32-compensated product path."""
    n_px = S * spec.n_pix
    out = torch.empty((S, spec.n_pix), dtype=torch.float32, device="cuda")
    ms_naive = time_extract(lya, torch, field, lya.ExtractParams(t_mode=0, precision=lya.PREC_F32_NAIVE), out, reps)
    ms_f64 = time_extract(lya, torch, field, lya.ExtractParams(t_mode=0, precision=lya.PREC_F64), out, max(2, reps // 4))
    del out
    res = {}
    for name, ms in (("f32_compensated", tau_ms_comp), ("f32_naive", ms_naive), ("f64", ms_f64)):
        res[name] = {"ms": ms, "px_per_s": n_px / (ms / 1e3), "fp32_pipe": fp32_pipe(pairs_px, n_px, ms, sms, clk_hz)}
    res["compensated_over_f64"] = ms_f64 / tau_ms_comp
    res["note"] = ("optical-depth kernel alone, same 65,536 x 4,096 field; f64 is the plain FP64 comparator kernel "
                   "(FP64 sums and exponentials, all pairs of the skewer's widest window); FP32-pipe fraction = "
                   "algorithmic pairs x 6 FP32 operations / duration / (SMs x 128 x max clock)")
    return res


def run_grid_object(lya, torch, steps, warmup, peaks, sms, clk_hz):
    """The 1536^3 grid (config 4): every one of its 2,359,296 rows x 1,536 px
    in one optical-depth launch, then the root-find and statistics, timed
    like the headline step."""
    spec, S, target = ls.GRID_1536, ls.GRID_1536_ROWS, ls.GRID_1536_FT
    rho, v, t = ls.grid_on_device(spec, S, torch)          # 43.5 GB on the device
    field = lya.Field(rho, v, t, box=spec.box, z=spec.z, borrow=True)
    params = lya.ExtractParams(t_mode=0)
    tau = torch.empty((S, spec.n_pix), dtype=torch.float32, device="cuda")
    F = torch.empty_like(tau)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        lya.extract_skewers(field, params, out=tau)
        A, _, st = lya.rescale_mean_flux_stats(tau, target, flux_out=F)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    clocks.start()
    for e in evs:
        e[0].record(stream)
        lya.extract_skewers(field, params, out=tau)
        e[1].record(stream)
        A, _, st = lya.rescale_mean_flux_stats(tau, target, flux_out=F)
        e[2].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = statistics.mean(e[0].elapsed_time(e[2]) for e in evs)
    tau_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    field.status()
    n_px = S * spec.n_pix
    r64, v64, t64 = ls.grid_rows(spec, np.arange(64))
    pairs_px = algorithmic_pairs_per_px(r64, v64, t64, lya.field_pixel_width(field))
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = ALG_BYTES_PER_PX * n_px / (tau_ms / 1e3) / 1e9
    per_row, profiled_hash = TAU_DRAM_PROFILE["grid1536"]
    mean_flux = fp64_mean_flux(torch, tau, A)
    field.close()
    del rho, v, t, tau, F
    torch.cuda.empty_cache()
    return {"workload": "grid_1536cubed_z2.3: all 2,359,296 rows x 1,536 px of a periodic 1536^3 grid "
                        "(1 h^-1 Gpc, T0 = 2e4 K, gamma = 1.4), one launch", "value": n_px / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms, "steps": steps, "A": A, "mean_flux": mean_flux,
            "stats_mean_flux": st.mean_flux, "target_mean_flux": target,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": per_row * S if tau_code_hash() == profiled_hash else None,
                         "kernel_ms": tau_ms, "alg_bytes_per_launch": ALG_BYTES_PER_PX * n_px},
            "pipes": {"alg_pairs_per_px": pairs_px,
                      "fp32_pipe": fp32_pipe(pairs_px, n_px, tau_ms, sms, clk_hz)},
            "clocks": clk, "parity": "tests/test_gpu_grid.py: 512 random rows (seed 1004) against the FP64 oracle",
            "l2": "inputs 43.5 GB > 129 MB L2: no flush between steps"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    grid = args.workload == "grid1536"
    spec = ls.GRID_1536 if grid else ls.GPC_4096
    S = (ls.GRID_1536_ROWS if grid else ls.GPC_4096_SKEWERS) if args.skewers is None else args.skewers
    target = ls.GRID_1536_FT if grid else ls.GPC_4096_FT
    if not grid:
        # host generation first: the spawn pool starts before any CUDA call
        rho, v, t = ls.skewers_parallel(spec, np.arange(S))
    import torch
    world, rank, local = dist_setup()
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4747_gb300 as lya

    stream = torch.cuda.current_stream()
    if grid:
        rho, v, t = ls.grid_on_device(spec, S, torch)       # 43.5 GB on the device
        field = lya.Field(rho, v, t, box=spec.box, z=spec.z, borrow=True)
    else:
        field = lya.Field(rho, v, t, box=spec.box, z=spec.z)
    params = lya.ExtractParams(t_mode=0, precision=lya.PREC_F32_COMPENSATED)
    tau = torch.empty((S, spec.n_pix), dtype=torch.float32, device="cuda")
    F = torch.empty_like(tau)
    n_px = S * spec.n_pix

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        lya.extract_skewers(field, params, out=tau)
        if ev is not None:
            ev[1].record(stream)
        A, _, st = lya.rescale_mean_flux_stats(tau, target, flux_out=F)
        return A, st

    for _ in range(args.warmup):
        A, st = step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    tau_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = lya.kernel_launches()
    start.record(stream)
    for k in range(args.steps):
        A, st = step(tau_ev[k])
    end.record(stream)
    end.synchronize()
    launches = lya.kernel_launches() - launches0
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = start.elapsed_time(end) / args.steps
    ms = max_over_ranks(ms, world)
    tau_ms = statistics.mean(a.elapsed_time(b) for a, b in tau_ev)

    # the mock-spectrum processing (Sec. 4) and the 1D flux power spectrum
    # (Sec. 5.3) on this step's F
    post = None
    if not grid and not args.no_post:
        post = run_post(lya, torch, field, F, S, spec, args.steps)

    # end to end through the public API: host inputs in, host flux out.  Two
    # device fields and two F buffers let step k+1's inputs cross to the device
    # (a loader thread, lya_field_load on its own stream) and step k-1's F
    # cross back (a copy stream) while step k computes.
    # algorithmic pairs of the sum per pixel, counted on 64 rows of the workload
    if grid:
        r64, v64, t64 = ls.grid_rows(spec, np.arange(64))
    else:
        r64, v64, t64 = rho[:64], v[:64], t[:64]
    pairs_px = algorithmic_pairs_per_px(r64, v64, t64, lya.field_pixel_width(field))
    del r64, v64, t64

    e2e = None
    if not args.no_e2e and not grid:
        e2e = run_e2e(lya, torch, field, spec, S, params, target, rho, v, t, tau, F,
                      max(3, min(args.steps, 8)), world, local)
        del rho, v, t
        # the host link bounds e2e: its measured bandwidth and e2e's use of it
        link = measure_link(torch)
        step_s = e2e["ms_per_step"] / 1e3
        e2e["link"] = link
        e2e["link_frac"] = {"h2d": e2e["h2d_bytes_per_step"] / step_s / 1e9 / link["h2d_gbs"],
                            "d2h": e2e["d2h_bytes_per_step"] / step_s / 1e9 / link["d2h_gbs"],
                            "note": "bytes per step / e2e time per step / the measured one-way bandwidth"}

    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = ALG_BYTES_PER_PX * n_px / (tau_ms / 1e3) / 1e9
    per_skewer, profiled_hash = TAU_DRAM_PROFILE[args.workload]
    same_kernel = tau_code_hash() == profiled_hash
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": per_skewer * S if same_kernel else None,
                "kernel": "tau_tile_kernel<compensated,8>", "kernel_ms": tau_ms,
                "peak_source": "measured" if peaks else "fallback",
                "alg_bytes_per_launch": ALG_BYTES_PER_PX * n_px}

    # the pair sum's arithmetic against the FP32 and MUFU (XU) pipe peaks at the
    # maximum SM clock: algorithmic pairs x FP32 operations per pair, one ex2 each
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk_hz = (peaks["sm_max_mhz"] if peaks else 2070.0) * 1e6
    pairs = pairs_px * n_px
    pipe_ncu, pipe_hash = TAU_PIPE_PROFILE.get(args.workload, (None, None))
    pipes = {"alg_pairs_per_px": pairs_px, "fp32_ops_per_pair": FP32_OPS_PER_PAIR,
             "fp32_achieved": pairs * FP32_OPS_PER_PAIR / (tau_ms / 1e3), "fp32_peak": sms * 128 * clk_hz,
             "fp32_frac": pairs * FP32_OPS_PER_PAIR / (tau_ms / 1e3) / (sms * 128 * clk_hz),
             "xu_achieved": pairs / (tau_ms / 1e3), "xu_peak": sms * 16 * clk_hz,
             "xu_frac": pairs / (tau_ms / 1e3) / (sms * 16 * clk_hz),
             "unit": "operations/s", "peak_clock_mhz": clk_hz / 1e6, "sms": sms,
             "ncu_pipe_pct": pipe_ncu if pipe_ncu and tau_code_hash() == pipe_hash else None}

    # A's defining property over all pixels, in FP64 (the root-find stops at
    # |<exp(-A tau)> - target| <= 1e-12)
    mean_flux = fp64_mean_flux(torch, tau, A)

    precision = None
    if not grid and not args.no_precision:
        precision = run_precision_variants(lya, torch, field, spec, S, tau_ms, pairs_px, sms, clk_hz,
                                           max(3, args.steps))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not grid:
        cpu = oracle_timing(spec, args.cpu_seconds)

    serving = None
    if not grid and not args.no_serving:
        del tau, F
        torch.cuda.empty_cache()
        serving = run_serving(lya, torch, 2.0, args.serve_seconds, burst=args.serve_burst,
                              budget=int(args.serve_budget_gb * (1 << 30)), peaks=peaks, sms=sms, clk_hz=clk_hz)
    field.close()

    grid_obj = None
    if not grid and not args.no_grid:
        torch.cuda.empty_cache()
        grid_obj = run_grid_object(lya, torch, max(3, min(args.steps, 5)), 2, peaks, sms, clk_hz)

    if rank == 0:
        line = {"metric": METRIC, "value": world * n_px / (ms / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(spec, S, {"parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                                                    "A": A, "mean_flux": mean_flux,
                                                    "mean_flux_definition": "<exp(-A tau)> over all pixels in FP64",
                                                    "stats_mean_flux": st.mean_flux}, grid),
                "roofline": roofline, "pipes": pipes, "precision_variants": precision, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk, "serving": serving, "grid1536": grid_obj,
                "post": post}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0



def run_serving_workload(args):
    """The served form alone: p50/p99 latency and served pixels/s."""
    import torch
    world, rank, local = dist_setup()
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4747_gb300 as lya
    clocks = ClockSampler(local)
    clocks.start()
    sv = run_serving(lya, torch, 5.0, 60.0, burst=args.serve_burst, budget=int(args.serve_budget_gb * (1 << 30)))
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": "served tau-skewer pixels/s, Poisson 200 req/s; p50/p99 latency", "value":
                sv["served_px_per_s"] * world, "unit": UNIT, "n_gpus": world, "steps": sv["steps"], "warmup": 5,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": {"workload": sv["workload"],
                                                               "parallelism": "replicas" if world > 1 else "1 GPU"},
                "latency_ms": {"p50": sv["p50_ms"], "p99": sv["p99_ms"]}, "serving": sv,
                "gpu_launches": sv["gpu_launches"], "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skewers", type=int, default=None, help="fewer skewers (debug only)")
    ap.add_argument("--workload", choices=["gpc", "grid1536", "serving"], default="gpc",
                    help="gpc: 65,536 x 4,096 px (the metric's workload); grid1536: all rows of a 1536^3 grid; "
                         "serving: 60 s of Poisson requests after 5 s of warm-up")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-post", action="store_true", help="skip the mock-spectrum and flux-power timings")
    ap.add_argument("--no-grid", action="store_true", help="skip the 1536^3 grid object of the default run")
    ap.add_argument("--no-precision", action="store_true", help="skip the naive and FP64 kernel timings")
    ap.add_argument("--serve-seconds", type=float, default=52.0,
                    help="measured seconds of the Poisson request stream in the default run (>= 10,000 requests)")
    ap.add_argument("--serve-burst", type=int, default=400, help="requests of the capacity burst")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0, help="serving memory budget (GiB)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
