"""The synthetic workloads of the benchmark follow their stated recipes (CPU only).

Batch (256 problems, seed 0): K ~ U{4..7}, J ~ U{4..8}, u0 = 0, g on the (2^J + 1) x (2^K - 1)^2
grid.  Serve: Poisson arrivals at 2000/s, square or L-shape with probability 1/2, K and J
independent with P(4 + k) proportional to 2^-k, k = 0..5.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_batch_workload_recipe():
    probs = bench.batch_workload(256, seed=0)
    assert len(probs) == 256
    Ks = np.array([p[0] for p in probs])
    Js = np.array([p[1] for p in probs])
    assert set(Ks) == {4, 5, 6, 7} and set(Js) == {4, 5, 6, 7, 8}
    for K, J, g, u0 in probs:
        assert g.shape == (2 ** J + 1, (2 ** K - 1) ** 2) and u0.shape == ((2 ** K - 1) ** 2,)
        assert not u0.any() and np.isfinite(g).all() and np.abs(g).max() > 0
    # the same seed gives the same problems
    again = bench.batch_workload(4, seed=0)
    for a, b in zip(probs[:4], again):
        assert a[:2] == b[:2] and np.array_equal(a[2], b[2])


def test_serve_arrivals_recipe():
    arr = bench.serve_arrivals(2000.0, 10.0, seed=0)
    n = len(arr)
    assert abs(n - 20000) < 5 * np.sqrt(20000)
    t = np.array([a[0] for a in arr])
    assert np.all(np.diff(t) > 0) and t[-1] <= 10.0
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000) < 0.05 / 2000
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05  # exponential: coefficient of variation 1
    dom = np.array([a[1] for a in arr])
    assert set(dom) == {0, 1} and abs(dom.mean() - 0.5) < 0.02
    pk = 2.0 ** -np.arange(6)
    pk /= pk.sum()
    for col in (2, 3):
        lev = np.array([a[col] for a in arr])
        freq = np.bincount(lev - 4, minlength=6) / n
        assert np.all(np.abs(freq - pk) < 5 * np.sqrt(pk * (1 - pk) / n)), freq
    # the default replay window of the benchmark
    assert len(bench.serve_arrivals(2000.0, 0.25, seed=0)) == 507
