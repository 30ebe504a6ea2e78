"""The serving loop on the GPU: each served request equals the same request
run alone, the library's direct path and, on small cases, the FP64 oracle;
admission by memory budget, release, continuous batching and errors.

Tolerances are those of the method (|F_a - F_b| <= 1e-5 absolute); results of
the same request in different mixes differ only by the summation order of
the shared-memory sort (about 1e-7).
"""
import threading
import time

import numpy as np
import pytest

import lya_synth as ls

pytestmark = pytest.mark.gpu

F_ATOL = 1e-5


@pytest.fixture(scope="module")
def lya():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4747_gb300 as lya
    return lya


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


# a pool with every skewer length, the extremes of the box range included
POOL = [(512, 1000.0), (1024, 300.0), (2048, 120.0), (4096, 1000.0), (8192, 50.0)]
POOL_SKEWERS = 192


@pytest.fixture(scope="module")
def pool(lya):
    fields, specs = [], []
    for k, (n, box) in enumerate(POOL):
        spec = ls.FieldSpec(n_pix=n, box=box, z=2.5, k_j=4.0, sigma_delta=1.5, T0=1.5e4, gamma=1.5,
                            seed=3000 + k)
        rho, v, _ = ls.skewers(spec, np.arange(POOL_SKEWERS), with_temp=False)
        fields.append(lya.Field(rho, v, None, box=box, z=spec.z))
        specs.append(spec)
    return fields, specs


def params(lya, T0, gamma):
    return lya.ExtractParams(t_mode=1, T0=T0, gamma=gamma)


def requests(n, seed, max_skewers=96):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        f = int(rng.integers(len(POOL)))
        m = int(np.clip(np.round(np.exp(rng.uniform(0, np.log(max_skewers)))), 1, max_skewers))
        ids = np.sort(rng.choice(POOL_SKEWERS, size=m, replace=False))
        out.append((f, ids, float(rng.uniform(1e4, 2.5e4)), float(rng.uniform(1.0, 1.6)),
                    float(rng.uniform(0.65, 0.85))))
    return out


def run_alone(lya, srv, fields, reqs):
    res = []
    for f, ids, T0, g, Ft in reqs:
        t = srv.submit(fields[f], params(lya, T0, g), ids, Ft)
        r = srv.wait(t, 120.0)
        assert r.done and r.status == 0, r
        res.append((r, srv.flux(t).cpu().numpy()))
        srv.release(t)
    return res


def run_mixed(lya, srv, fields, reqs):
    tickets = [srv.submit(fields[f], params(lya, T0, g), ids, Ft) for f, ids, T0, g, Ft in reqs]
    res = []
    for t in tickets:
        r = srv.wait(t, 300.0)
        assert r.done and r.status == 0, r
        res.append((r, srv.flux(t).cpu().numpy()))
    for t in tickets:
        srv.release(t)
    return res


def test_alone_and_mixed_agree(lya, pool):
    fields, _ = pool
    reqs = requests(24, seed=5)
    with lya.Server(budget_bytes=4 << 30, max_slots=64) as srv:
        alone = run_alone(lya, srv, fields, reqs)
        mixed = run_mixed(lya, srv, fields, reqs)
        info = srv.info()
    assert info["completed"] == 2 * len(reqs) and info["failed"] == 0
    assert info["arena_used"] == 0
    worst = 0.0
    for (ra, Fa), (rm, Fm) in zip(alone, mixed):
        assert Fa.shape == Fm.shape
        d = float(np.abs(Fa - Fm).max())
        worst = max(worst, d)
        assert d <= F_ATOL
        assert rm.A == pytest.approx(ra.A, rel=1e-5)
        assert ra.stats.n == rm.stats.n
        assert rm.stats.mean_flux == pytest.approx(ra.stats.mean_flux, abs=1e-6)
    print(f"max |F_alone - F_mixed| = {worst:.2e}")


def test_served_equals_direct_path(lya, pool):
    """Served F, A and statistics against extract_skewers + rescale_mean_flux + flux_stats."""
    import torch
    fields, _ = pool
    reqs = requests(10, seed=9)
    with lya.Server(budget_bytes=2 << 30, max_slots=16) as srv:
        tickets = [srv.submit(fields[f], params(lya, T0, g), ids, Ft) for f, ids, T0, g, Ft in reqs]
        for t, (f, ids, T0, g, Ft) in zip(tickets, reqs):
            r = srv.wait(t, 120.0)
            assert r.done and r.status == 0
            Fs = srv.flux(t)
            tau = lya.extract_skewers(fields[f], params(lya, T0, g), ids=torch.as_tensor(ids))
            A, F = lya.rescale_mean_flux(tau, Ft)
            assert r.A == pytest.approx(A, rel=1e-5)
            assert float((Fs - F).abs().max()) <= F_ATOL
            st = lya.flux_stats(Fs)
            assert np.array_equal(st.pdf, r.stats.pdf)           # same F values, exact bins
            assert r.stats.n == st.n == ids.size * fields[f].n_pix
            assert r.stats.mean_flux == pytest.approx(st.mean_flux, abs=1e-8)   # FP32 partial sums
            # the mean of the FP32 F values: A is the root of the exact mean
            # (to 1e-12), F is written with the MUFU exponential, whose small
            # bias (~1e-8) shows here
            assert r.stats.mean_flux == pytest.approx(Ft, abs=1e-7)
            assert r.stats.var_flux == pytest.approx(st.var_flux, rel=1e-6)
            srv.release(t)


def test_served_matches_oracle(lya, orc, pool):
    """Small served requests against the FP64 oracle (power-law T, Eq. 4-6, Sec. 2.3)."""
    fields, specs = pool
    cases = [(0, [0, 5, 17], 1.2e4, 1.1, 0.7), (1, [3, 4], 2.4e4, 1.55, 0.82), (2, [7], 1.8e4, 1.3, 0.75)]
    with lya.Server(budget_bytes=1 << 30, max_slots=8) as srv:
        tickets = [srv.submit(fields[f], params(lya, T0, g), np.array(ids), Ft) for f, ids, T0, g, Ft in cases]
        for t, (f, ids, T0, g, Ft) in zip(tickets, cases):
            r = srv.wait(t, 120.0)
            assert r.done and r.status == 0
            Fs = srv.flux(t).cpu().numpy().astype(np.float64)
            spec = specs[f]
            rho, v, _ = ls.skewers(spec, np.array(ids), with_temp=False)
            p = orc.Params(box=spec.box, z=spec.z, h=0.72, omega_m=0.26, omega_l=0.74, omega_b=0.0444,
                           y_he=0.24, t_mode=1, T0=T0, gamma=g, delta_pivot=10.0, gamma12=1.0)
            tau = orc.tau(p, rho, v)
            A, _ = orc.rescale(tau, Ft)
            Fo = orc.flux(tau, A)
            assert float(np.abs(Fs - Fo).max()) <= F_ATOL
            assert r.A == pytest.approx(A, rel=1e-4)
            srv.release(t)


def test_short_request_overtakes_long_one(lya):
    """Continuous batching: a short request submitted while a long one runs
    is admitted in the next step and finishes first."""
    spec = ls.FieldSpec(n_pix=8192, box=50.0, z=2.5, k_j=4.0, sigma_delta=1.5, T0=1.5e4, gamma=1.5, seed=77)
    rho, v, _ = ls.skewers(spec, np.arange(1024), with_temp=False)
    big = lya.Field(rho, v, None, box=spec.box, z=spec.z)
    s2 = ls.FieldSpec(n_pix=512, box=500.0, z=2.5, k_j=4.0, sigma_delta=1.5, T0=1.5e4, gamma=1.5, seed=78)
    r2, v2, _ = ls.skewers(s2, np.arange(8), with_temp=False)
    small = lya.Field(r2, v2, None, box=s2.box, z=s2.z)
    with lya.Server(budget_bytes=2 << 30, max_slots=8, step_target_us=500.0) as srv:
        tb = srv.submit(big, params(lya, 2.0e4, 1.5), np.arange(1024), 0.75)
        time.sleep(0.002)
        ts = srv.submit(small, params(lya, 1.5e4, 1.3), np.arange(8), 0.8)
        rs = srv.wait(ts, 120.0)
        rb = srv.wait(tb, 120.0)
        assert rs.done and rb.done and rs.status == 0 and rb.status == 0
        assert rs.t_done_ns < rb.t_done_ns
        assert rs.t_admit_ns < rb.t_done_ns               # admitted while the long one was on the GPU
        assert srv.info()["steps"] >= 3
        srv.release(ts)
        srv.release(tb)


def test_budget_admission_and_release(lya, pool):
    fields, _ = pool
    f = fields[3]                                           # 4096 px: 32 KiB of tau + F per skewer
    per_skewer = 2 * 4 * f.n_pix
    budget = 64 * per_skewer                                # 2 MiB: one 48-skewer request at a time
    with lya.Server(budget_bytes=budget, max_slots=8) as srv:
        with pytest.raises(lya.LyaError) as e:
            srv.submit(f, params(lya, 1.5e4, 1.5), np.arange(POOL_SKEWERS), 0.8)   # never fits
        assert e.value.status == -6
        t1 = srv.submit(f, params(lya, 1.5e4, 1.5), np.arange(48), 0.8)
        t2 = srv.submit(f, params(lya, 1.5e4, 1.5), np.arange(48, 96), 0.8)       # waits for t1's memory
        r1 = srv.wait(t1, 60.0)
        assert r1.done and r1.status == 0
        time.sleep(0.2)
        assert not srv.poll(t2).done                         # t1's F still holds the arena
        info = srv.info()
        assert info["queued"] == 1 and info["arena_used"] > 0
        with pytest.raises(lya.LyaError):
            srv.release(t2)                                  # not finished
        srv.release(t1)
        r2 = srv.wait(t2, 60.0)
        assert r2.done and r2.status == 0
        srv.release(t2)
        assert srv.info()["arena_used"] == 0


def test_field_is_held_while_requested(lya, pool):
    fields, specs = pool
    spec = specs[3]                                         # 4096 px: 24 skewers hold 768 KiB
    rho, v, _ = ls.skewers(spec, np.arange(24), with_temp=False)
    f = lya.Field(rho, v, None, box=spec.box, z=spec.z)
    with lya.Server(budget_bytes=1 << 20, max_slots=4) as srv:
        t1 = srv.submit(fields[3], params(lya, 1.5e4, 1.5), np.arange(24), 0.8)
        r1 = srv.wait(t1, 60.0)
        assert r1.done
        t2 = srv.submit(f, params(lya, 1.5e4, 1.5), np.arange(24), 0.8)  # queued behind t1's F
        time.sleep(0.1)
        assert not srv.poll(t2).done
        st = lya.load_library().lya_destroy_field(f.handle)
        assert st == -8                                       # LYA_EBUSY
        srv.release(t1)
        assert srv.wait(t2, 60.0).status == 0
        srv.release(t2)
    f.close()


def test_submit_errors_and_failed_requests(lya, pool):
    fields, _ = pool
    with lya.Server(budget_bytes=1 << 28, max_slots=4) as srv:
        for bad in (dict(ids=[POOL_SKEWERS]), dict(ids=[-1]), dict(target=1.0), dict(target=0.0)):
            kw = dict(ids=[0, 1], target=0.8)
            kw.update(bad)
            with pytest.raises(lya.LyaError):
                srv.submit(fields[0], params(lya, 1.5e4, 1.5), kw["ids"], kw["target"])
        p = params(lya, 1.5e4, 1.5)
        p.precision = lya.PREC_F32_NAIVE
        with pytest.raises(lya.LyaError):
            srv.submit(fields[0], p, [0], 0.8)
        # a field with no absorbers: no A reaches the target -> the request fails, the server goes on
        z = lya.Field(np.zeros((4, 512), np.float32), np.zeros((4, 512), np.float32), None, box=100.0, z=2.5)
        t = srv.submit(z, params(lya, 1.5e4, 1.5), [0, 1, 2, 3], 0.8)
        r = srv.wait(t, 60.0)
        assert r.done and r.status in (-1, -4) and r.flux_ptr == 0
        srv.release(t)
        t = srv.submit(fields[0], params(lya, 1.5e4, 1.5), [0, 1], 0.8)
        assert srv.wait(t, 60.0).status == 0
        srv.release(t)
        info = srv.info()
        assert info["failed"] == 1 and info["completed"] == 1


def test_autotune_and_concurrent_clients(lya, pool):
    """Autotune every skewer length, then four client threads submit at once."""
    fields, _ = pool
    with lya.Server(budget_bytes=2 << 30, max_slots=32) as srv:
        for f in fields:
            shift = srv.autotune(f, params(lya, 1.5e4, 1.5), max_rows=128)
            assert 0 <= shift <= 3
        shifts = srv.info()["group_shift"]
        assert sum(1 for s in shifts if s >= 0) == len(fields)
        reqs = requests(32, seed=21, max_skewers=32)
        results = [None] * len(reqs)

        def client(k):
            for i in range(k, len(reqs), 4):
                f, ids, T0, g, Ft = reqs[i]
                t = srv.submit(fields[f], params(lya, T0, g), ids, Ft)
                r = srv.wait(t, 120.0)
                results[i] = (r.status, r.done)
                srv.release(t)

        threads = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert all(r == (0, True) for r in results)
    # tuning needs an idle server: a request held in the queue keeps it busy
    f = fields[3]
    with lya.Server(budget_bytes=1 << 20, max_slots=4) as srv:
        t1 = srv.submit(f, params(lya, 1.5e4, 1.5), np.arange(24), 0.8)
        assert srv.wait(t1, 60.0).status == 0
        t2 = srv.submit(f, params(lya, 1.5e4, 1.5), np.arange(24, 48), 0.8)    # waits for memory
        with pytest.raises(lya.LyaError) as e:
            srv.autotune(f, params(lya, 1.5e4, 1.5))
        assert e.value.status == -8
        srv.release(t1)
        assert srv.wait(t2, 60.0).status == 0
        srv.release(t2)
