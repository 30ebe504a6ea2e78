"""The optical-depth kernel's shared-memory indices, checked.

The library is built a second time with -DLYA_CHECKED: before every
shared-memory index of the tile gather is used (target bins, record
positions, seam copies, run searches, tile order, record ranges) the kernel
checks it and, on a failure, sets bit 2 of the launch's error word instead of
trapping.  A separate process loads that build and runs the geometries that
take every path of the kernel: local runs with seam copies, runs split at a
crowded seam, tiles whose run spans the whole skewer, envelope scans for wide
windows with four-pixel lanes, lengths that are not a multiple of four, the
pixel-averaged profile, the exponential variants, the plain sum and a served
request.  No check may fail (the field's error word stays clear).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import os, sys
import numpy as np
import torch
sys.path.insert(0, os.getcwd())
import lya_synth as ls
import paper_1105_4747_gb300 as lya
assert lya.library_path() == os.environ["LYA_LIBRARY"]
lya.load_library()
torch.cuda.set_device(0)

def run(spec, rho, v, t, params, name):
    f = lya.Field(rho, v, t, box=spec.box, z=spec.z)
    tau = lya.extract_skewers(f, params)
    torch.cuda.synchronize()
    f.status()                                   # raises if any check failed
    assert bool(torch.isfinite(tau).all()), name
    f.close()
    print("ok", name, flush=True)

tiny = ls.TINY_20MPC
r, v, t = ls.skewers(tiny, np.arange(16))
for prec in (0, 1):
    run(tiny, r, v, t, lya.ExtractParams(precision=prec), f"tiny prec {prec}")
run(tiny, r, v, t, lya.ExtractParams(profile=lya.PROFILE_AVERAGED), "tiny averaged")

gpc = ls.GPC_4096
r, v, t = ls.skewers(gpc, np.arange(64))
run(gpc, r, v, t, lya.ExtractParams(), "gpc 64 skewers")
run(gpc, r, v, t, lya.ExtractParams(profile=lya.PROFILE_AVERAGED), "gpc averaged")

N = 256
probe = lya.Field(np.ones((1, N), np.float32), np.zeros((1, N), np.float32), np.full((1, N), 1.5e4, np.float32),
                  box=tiny.box, z=tiny.z)
du = lya.field_pixel_width(probe)                 # km/s per pixel
probe.close()
j = np.arange(N, dtype=np.float64)
for target in (0, N - 1):
    rho = np.ones((2, N), np.float32)
    vv = np.stack([(target - j) * du, (target - j) * du + 0.3 * du * np.sin(j)]).astype(np.float32)
    tt = np.full((2, N), 1.5e4, np.float32)
    run(tiny, rho, vv, tt, lya.ExtractParams(), f"seam crowd {target}")

for n_pix in (18, 258, 1030):
    sp = tiny.with_(n_pix=n_pix, box=20.0 * n_pix / 256, seed=13)
    r, v, t = ls.skewers(sp, np.arange(4))
    run(sp, r, v, t, lya.ExtractParams(), f"n_pix {n_pix}")

wide = gpc.with_(n_pix=8192, box=50.0, T0=2.5e4, gamma=1.6, seed=11)
r, v, _ = ls.skewers(wide, np.arange(3), with_temp=False)
for m in (lya.EXP_MUFU, lya.EXP_RECURRENCE, lya.EXP_POLY_SPLIT):
    run(wide, r, v, None, lya.ExtractParams(t_mode=1, T0=2.5e4, gamma=1.6, exp_method=m), f"wide exp {m}")

f = lya.Field(r, v, None, box=wide.box, z=wide.z)
ids = np.arange(3)
with lya.Server(budget_bytes=1 << 28, max_slots=4) as srv:
    tk = srv.submit(f, lya.ExtractParams(t_mode=1, T0=2.5e4, gamma=1.6), ids, 0.8)
    res = srv.wait(tk, 120.0)
    assert res.done and res.status == 0, res.status
    srv.release(tk)
f.status()
f.close()
print("ok served", flush=True)
print("checked ok", flush=True)
'''


def test_checked_build_sees_no_out_of_bounds_index():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_4747_gb300 import build as lib_build
    path = lib_build.build(checked=True)
    env = dict(os.environ, LYA_LIBRARY=path)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout
