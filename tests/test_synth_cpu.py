"""Input generators of the served workload: the recipe's stated properties
(sizes, mix fractions, in-block edge fraction, mean degree, bounds)."""
import numpy as np

import synth


def test_serve_specs_recipe():
    sp = synth.serve_specs(20_000, seed=5)
    ns = np.array([s[2] for s in sp])
    assert ns.min() >= 100 and ns.max() <= 2_000_000
    # log-uniform: the median is near the geometric mean of the bounds
    assert abs(np.log(np.median(ns)) - 0.5 * (np.log(100) + np.log(2e6))) < 0.1
    assert abs(np.mean([s[0] == "louvain" for s in sp]) - 0.7) < 0.015
    assert abs(np.mean([s[1] == "rmat" for s in sp]) - 0.5) < 0.015
    ks = np.array([s[3] for s in sp])
    assert ks.min() == 2 and ks.max() == 50
    assert sp == synth.serve_specs(20_000, seed=5)  # seeded


def test_sbm_sparse_properties():
    n, k = 30_000, 6
    g = synth.sbm_sparse(n, k, 16, seed=2)
    off, cols = g.off.numpy(), g.cols.numpy()
    rows = np.repeat(np.arange(n), np.diff(off))
    assert (rows != cols).all()
    assert 15.5 < len(cols) / n <= 16.0          # few duplicates or loops dropped
    s = n // k
    expect_in = 100 * (s - 1) / (100 * (s - 1) + n - s)
    frac_in = (g.planted[rows] == g.planted[cols]).mean()
    assert abs(frac_in - expect_in) < 0.01
    # symmetric, sorted rows
    keys = rows.astype(np.int64) * n + cols
    assert (np.sort(keys) == keys).all()
    assert np.array_equal(np.sort(cols.astype(np.int64) * n + rows), keys)


def test_rmat_n_bounds_and_symmetry():
    for n in (100, 1000, 1025):
        g = synth.rmat_n(n, 8, seed=3)
        off, cols = g.off.numpy(), g.cols.numpy()
        assert g.n == n and len(off) == n + 1 and (cols < n).all() and (cols >= 0).all()
        rows = np.repeat(np.arange(n), np.diff(off))
        keys = rows.astype(np.int64) * n + cols
        assert np.array_equal(np.sort(cols.astype(np.int64) * n + rows), keys)
        assert (rows != cols).all()
