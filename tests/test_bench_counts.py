"""Host-side figures bench.py reports, checked without a GPU.

The `pipes` object counts the algorithmic pairs of the Eq. 6 sum,
#{(i, j): |v_H(i) - u_j| <= 8 b_j} with v_H(i) = i du and u_j = j du + v_j
at the nearest periodic image, per output pixel, from interval arithmetic on
each source.  Here that count is checked against the pairs enumerated one by
one on small skewers.
"""
import numpy as np

import bench
import lya_synth as ls


def brute_pairs(rho, v, t, du, window=8.0):
    N = rho.shape[1]
    i = np.arange(N, dtype=np.float64)
    n = 0
    for r in range(rho.shape[0]):
        for j in range(N):
            if not rho[r, j] > 0:
                continue
            b = np.sqrt(2.0 * bench.KB_J_PER_K * float(t[r, j]) / bench.M_H_KG) / 1e3
            u = j * du + float(v[r, j])
            V = N * du
            d = np.mod(i * du - u + 0.5 * V, V) - 0.5 * V      # nearest periodic image, [-V/2, V/2)
            n += int(np.count_nonzero(np.abs(d) <= window * b))
    return n / rho.size


def test_pair_count_matches_enumeration():
    spec = ls.TINY_20MPC
    rho, v, t = ls.skewers(spec, np.arange(3))
    rho = rho.copy()
    rho[1, ::7] = 0.0                       # sources with no gas take no pairs
    for du in (7.7, 2.0, 31.0):                # windows well inside half the box
        got = bench.algorithmic_pairs_per_px(rho, v, t, du)
        want = brute_pairs(rho, v, t, du)
        assert abs(got - want) <= 1e-12 * max(1.0, want), (du, got, want)


def test_pair_count_of_one_line():
    # one source at rest on pixel 10, b = 10 km/s, du = 5 km/s: 8b = 80 km/s
    # covers pixels 10 +- 16, 33 pixels
    N = 64
    rho = np.zeros((1, N)); rho[0, 10] = 1.0
    v = np.zeros((1, N))
    T = 1e4 * (10.0 / (np.sqrt(2.0 * bench.KB_J_PER_K * 1e4 / bench.M_H_KG) / 1e3)) ** 2
    t = np.full((1, N), T)
    assert bench.algorithmic_pairs_per_px(rho, v, t, 5.0) * N == 33.0
