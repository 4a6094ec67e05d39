"""Pins of the oracle's toy generator (CPU).

- Philox4x64-10 against numpy's Philox bit generator (the same published
  algorithm, Salmon et al. SC'11; numpy advances the counter by one before
  each block).
- The inverse complementary error function against scipy.
- Every leaf's sampler: Kolmogorov-Smirnov distance between 100k drawn values
  and the CDF of the oracle's normalised density (itself pinned by quadrature
  in test_oracle_pins.py), integrated numerically on a fine grid.
- Component structure and support: counts per component in order, values of
  FP32 columns inside the range (ARGUS strictly below m0)."""
import numpy as np
import pytest

import datagen
import oracle


def test_philox_matches_numpy():
    rng = np.random.default_rng(0)
    for _ in range(20):
        key = [int(x) for x in rng.integers(0, 2**63, 2)]
        ctr = [int(x) for x in rng.integers(0, 2**62, 4)]
        bg = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
        want = [int(x) for x in bg.random_raw(4)]
        ctr1 = list(ctr)
        ctr1[0] += 1
        assert oracle.philox4x64(ctr1, key) == want


def test_erfcinv_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    qs = np.concatenate([np.logspace(-300, -1, 60), np.linspace(0.01, 1.99, 199),
                         2 - np.logspace(-15, -1, 30)])
    for q in qs:
        want = sp.erfcinv(q)
        assert abs(oracle.erfcinv(q) - want) <= 2e-15 * max(abs(want), 1e-300), q
    assert oracle.erfcinv(1.0) == 0.0


def single(kind, params, lo, hi):
    return {"obs": [(lo, hi)], "params": list(params),
            "nodes": [{"type": kind, "obs": 0, "params": list(range(len(params)))}],
            "root": 0}


def cdf_grid(kind, params, lo, hi, n=100_001):
    x = np.linspace(lo, hi, n)
    f = np.array([np.exp(oracle.leaf_logf(kind, params, lo, hi, xi)[0]) for xi in x])
    c = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(x))])
    return x, c / c[-1]


CASES = [
    ("gauss", [5.0, 0.5], 0.0, 10.0),
    ("gauss", [0.3, 1.2], 1.0, 4.0),          # only the upper tail
    ("gauss", [0.3, 1.2], -4.0, -1.5),        # only the lower tail
    ("exp", [-0.3], 0.0, 10.0),
    ("exp", [0.8], 0.0, 10.0),
    ("cheb", [0.2, -0.1, 0.05, 0.02], -1.0, 1.0),
    ("cb", [5.279, 0.003, 1.5, 3.0], 5.20, 5.29),
    ("cb", [0.0, 1.0, -1.2, 1.0], -3.0, 12.0),  # high-side tail, n = 1
    ("argus", [5.29, -20.0, 0.5], 5.20, 5.29),
    ("argus", [5.29, 2.0, 0.5], 5.0, 5.29),     # c > 0
    ("johnson", [0.5, 1.3, -0.4, 1.7], -2.0, 3.0),
    ("johnson", [0.0, 1.0, 2.5, 0.9], 2.0, 40.0),  # far upper tail only
]


@pytest.mark.parametrize("kind,params,lo,hi", CASES)
def test_leaf_sampler_distribution(kind, params, lo, hi):
    n = 100_000
    spec = single(kind, params, lo, hi)
    if kind == "argus":
        spec["fixed"] = [True, False, True]
    cols, ex, rc = oracle.generate(spec, [params], [[n]], [0, n], seed=20031287, col_f32=False)
    assert rc == 0 and ex == 0
    x = np.sort(cols[0])
    assert x[0] >= lo and x[-1] <= hi
    gx, gc = cdf_grid(kind, params, lo, hi)
    F = np.interp(x, gx, gc)
    i = np.arange(1, n + 1)
    d = max(np.max(i / n - F), np.max(F - (i - 1) / n))
    assert d * np.sqrt(n) < 1.8, (kind, params, d * np.sqrt(n))


def test_components_in_order_and_fp32_support():
    spec = datagen.cb_argus_spec()
    p = list(spec["params"])
    counts = np.array([[300, 4000], [0, 7], [5, 0]])
    off = np.concatenate([[0], np.cumsum(counts.sum(1))])
    cols, ex, rc = oracle.generate(spec, [p] * 3, counts, off, seed=7, col_f32=True)
    assert rc == 0 and ex == 0
    x = cols[0]
    assert np.all(x == x.astype(np.float32))
    assert np.all((x >= 5.20) & (x < 5.29))
    # the Crystal Ball block peaks at m0 = 5.279; the ARGUS block is broad
    assert abs(np.median(x[:300]) - 5.279) < 0.002
    assert 5.21 < np.median(x[300:4300]) < 5.27
    assert abs(np.median(x[4300:4307]) - 5.24) < 0.05 and abs(np.median(x[4307:]) - 5.279) < 0.01
    # seeded: the same call gives the same events, another seed others
    again, _, _ = oracle.generate(spec, [p] * 3, counts, off, seed=7, col_f32=True)
    other, _, _ = oracle.generate(spec, [p] * 3, counts, off, seed=8, col_f32=True)
    assert np.array_equal(again, cols) and not np.array_equal(other, cols)
