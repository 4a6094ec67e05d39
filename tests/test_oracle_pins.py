"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to an independent source: a library
implementation of the same density (scipy.stats / numpy.polynomial), brute-force
quadrature (mpmath), a closed form from sufficient statistics, an invariant of
maximum likelihood, or finite differences of a quantity that is itself pinned.
A plausible slip in the oracle -- a dropped term, a wrong sign, a swapped
parameter -- fails at least one of them.
"""
import math

import mpmath as mp
import numpy as np
import pytest
import scipy.stats as st
from numpy.polynomial import chebyshev as npcheb

import datagen
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- references

def lib_logpdf(kind, th, lo, hi, x):
    """log of the normalised density on [lo, hi] from an independent library."""
    x = np.asarray(x, np.float64)
    if kind == "gauss":
        mu, s = th
        return st.truncnorm((lo - mu) / s, (hi - mu) / s, loc=mu, scale=s).logpdf(x)
    if kind == "exp":
        (lam,) = th
        L = hi - lo
        if lam < 0:
            return st.truncexpon(L * -lam, loc=lo, scale=1 / -lam).logpdf(x)
        return st.truncexpon(L * lam, loc=0.0, scale=1 / lam).logpdf(hi - x)
    if kind == "cheb":
        poly = npcheb.Chebyshev([1.0, *th])
        u = (2 * x - lo - hi) / (hi - lo)
        anti = poly.integ()
        integral = 0.5 * (hi - lo) * (anti(1.0) - anti(-1.0))
        return np.log(poly(u) / integral)
    if kind == "cb":
        m0, s, a, n = th
        if a > 0:
            d = st.crystalball(a, n, loc=m0, scale=s)
            return d.logpdf(x) - np.log(d.cdf(hi) - d.cdf(lo))
        d = st.crystalball(-a, n, loc=-m0, scale=s)
        return d.logpdf(-x) - np.log(d.cdf(-lo) - d.cdf(-hi))
    if kind == "argus":
        m0, c, p = th
        assert p == 0.5
        d = st.argus(math.sqrt(-2 * c), loc=0.0, scale=m0)
        return d.logpdf(x) - np.log(d.cdf(min(hi, m0)) - d.cdf(lo))
    if kind == "johnson":
        mu, lam, gamma, delta = th
        d = st.johnsonsu(gamma, delta, loc=mu, scale=lam)
        return d.logpdf(x) - np.log(d.cdf(hi) - d.cdf(lo))
    raise KeyError(kind)


def oracle_lognorm(kind, th, lo, hi, x):
    I, _, rc = oracle.leaf_norm(kind, th, lo, hi)
    assert rc == 0
    out = []
    for xi in np.atleast_1d(x):
        lf, _, rc = oracle.leaf_logf(kind, th, lo, hi, float(xi))
        assert rc == 0
        out.append(lf - math.log(I))
    return np.array(out)


def fd_step(kind, th, j, lo, hi, rel):
    """Difference step on the natural scale of parameter j: the width for a
    location parameter, the parameter itself otherwise."""
    if kind in ("gauss", "cb", "johnson") and j == 0:
        return rel * th[1]
    if kind == "argus" and j == 0:
        return rel * (hi - lo)
    if kind == "cb" and j == 3 and abs(th[3] - 1.0) < 1e-2:
        return rel
    return rel * max(abs(th[j]), 1e-2)


def richardson(f, x, h):
    """Central difference with one Richardson step: O(h^4)."""
    d1 = (f(x + h) - f(x - h)) / (2 * h)
    d2 = (f(x + h / 2) - f(x - h / 2)) / h
    return (4 * d2 - d1) / 3


LEAF_CASES = [
    ("gauss", [0.25, 1.1], -10.0, 10.0),
    ("gauss", [5.0, 0.5], 0.0, 10.0),
    ("gauss", [0.0, 1.0], 3.0, 4.0),            # far tail, erfc branch
    ("gauss", [0.0, 1.0], -4.5, -3.0),          # far left tail
    ("exp", [-0.3], 0.0, 10.0),
    ("exp", [-0.5], 0.0, 10.0),
    ("exp", [0.7], -1.0, 2.0),
    ("exp", [2e-4], 0.0, 3.0),                  # series branch of <x>
    ("cheb", [0.2, -0.1, 0.05, 0.02], -1.0, 1.0),
    ("cheb", [0.3, 0.1], 2.0, 7.0),
    ("cheb", [-0.2, 0.1, 0.1, -0.05, 0.02, 0.01], -3.0, 5.0),
    ("cb", [5.279, 0.003, 1.5, 3.0], 5.20, 5.29),
    ("cb", [0.0, 1.0, 1.0, 2.5], -5.0, 5.0),
    ("cb", [0.0, 1.0, -1.2, 4.0], -5.0, 6.0),   # high-side tail
    ("cb", [0.0, 1.0, 0.8, 1.0], -6.0, 3.0),    # n = 1: log form
    ("cb", [0.0, 1.0, 0.8, 1.0000004], -6.0, 3.0),
    ("cb", [0.0, 1.0, 2.0, 5.0], 1.0, 3.0),     # core only
    ("cb", [0.0, 1.0, 2.0, 5.0], -9.0, -3.0),   # tail only
    ("argus", [5.29, -20.0, 0.5], 5.20, 5.29),
    ("argus", [5.29, -1.0, 0.5], 5.0, 5.29),    # series branch
    ("argus", [1.0, -40.0, 0.5], 0.2, 0.9),     # range ends below m0
    ("argus", [1.0, -3.0, 0.5], 0.0, 1.5),      # range extends past m0
    ("argus", [5.29, -20.0, 0.8], 5.20, 5.29),  # p other than 1/2
    ("argus", [1.0, -3.0, 1.0], 0.0, 1.5),
    ("argus", [1.0, 4.0, 2.5], 0.2, 0.9),       # c > 0, range below m0
    ("argus", [1.0, -30.0, 0.3], 0.5, 1.0),
    ("johnson", [0.5, 1.3, -0.4, 1.7], -2.0, 3.0),
    ("johnson", [5.28, 0.004, 0.8, 1.1], 5.20, 5.29),   # heavy tails, skewed
    ("johnson", [0.0, 1.0, 0.0, 3.0], -1.0, 8.0),       # near-Gaussian core
    ("johnson", [0.0, 1.0, 2.5, 0.9], 2.0, 40.0),       # far upper tail only
]


@pytest.mark.parametrize("kind,th,lo,hi", LEAF_CASES)
def test_normalised_leaf_matches_library_density(kind, th, lo, hi):
    if kind == "cb" and th[3] <= 1.0 + 1e-3:
        pytest.skip("scipy's full-line Crystal Ball is improper for n <= 1; "
                    "this case is pinned by quadrature")
    if kind == "argus" and th[2] != 0.5:
        pytest.skip("scipy's ARGUS has p = 1/2; other p are pinned by quadrature and, "
                    "for p = 1, by the closed form")
    top = min(hi, th[0]) if kind == "argus" else hi
    xs = np.linspace(lo, top, 23)[1:-1]
    want = lib_logpdf(kind, th, lo, hi, xs)
    got = oracle_lognorm(kind, th, lo, hi, xs)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-11)


def _kinks(kind, th, lo, hi):
    pts = [lo, hi]
    if kind == "cb":
        m0, s, a, _ = th
        k = m0 - s * a if a > 0 else m0 - s * a
        pts.append(k)
    if kind == "argus":
        pts.append(th[0])
    return sorted(p for p in set(pts) if lo <= p <= hi)


@pytest.mark.parametrize("kind,th,lo,hi", LEAF_CASES + [
    ("gauss", [0.3, 1.2], 0.3 - 0.12, 0.3 + 0.36),       # tiny ranges
    ("cb", [0.0, 1.0, 1.0, 3.0], -1.2, -0.7),            # straddles -alpha
    ("argus", [1.0, -10.0, 0.5], 0.98, 1.0),             # up to m0
    ("argus", [1.0, 2.0, 0.5], 0.1, 1.0),                # c > 0: series only
    ("argus", [1.0, 0.0, 0.5], 0.1, 1.0),                # c = 0
    ("exp", [0.0], -2.0, 3.0),
])
def test_norm_equals_quadrature(kind, th, lo, hi):
    mp.mp.dps = 30

    def f(x):
        lf, _, _ = oracle.leaf_logf(kind, th, lo, hi, float(x))
        return mp.e ** mp.mpf(lf) if lf > -1e300 else mp.mpf(0)
    quad = mp.quad(f, _kinks(kind, th, lo, hi))
    I, _, rc = oracle.leaf_norm(kind, th, lo, hi)
    assert rc == 0
    assert abs(I - float(quad)) <= 1e-12 * abs(float(quad))


@pytest.mark.parametrize("kind,th,lo,hi", LEAF_CASES + [
    ("argus", [1.0, 2.0, 0.5], 0.1, 1.0), ("exp", [0.0], -2.0, 3.0)])
def test_norm_derivatives_match_differences(kind, th, lo, hi):
    I, dI, rc = oracle.leaf_norm(kind, th, lo, hi)
    assert rc == 0
    for j in range(len(th)):
        h = fd_step(kind, th, j, lo, hi, 2e-4)

        def I_of(v):
            t = list(th)
            t[j] = v
            return oracle.leaf_norm(kind, t, lo, hi)[0]
        if kind == "argus" and j == 0 and th[0] >= hi:
            # b' = min(hi, m0) switches at m0 = hi, where I has a square-root
            # kink: difference from the left only (5-point one-sided stencil)
            x = th[0]
            fd = (25 * I_of(x) - 48 * I_of(x - h) + 36 * I_of(x - 2 * h)
                  - 16 * I_of(x - 3 * h) + 3 * I_of(x - 4 * h)) / (12 * h)
        else:
            fd = richardson(I_of, th[j], h)
        assert abs(dI[j] - fd) <= 1e-8 * max(abs(fd), 1e-3 * abs(I)), (j, dI[j], fd)


@pytest.mark.parametrize("kind,th,lo,hi", LEAF_CASES)
def test_logf_derivatives_match_differences(kind, th, lo, hi):
    top = min(hi, th[0]) if kind == "argus" else hi
    for x in np.linspace(lo, top, 9)[1:-1]:
        _, d, rc = oracle.leaf_logf(kind, th, lo, hi, float(x))
        for j in range(len(th)):
            h = fd_step(kind, th, j, lo, hi, 1e-4)

            def lf(v):
                t = list(th)
                t[j] = v
                return oracle.leaf_logf(kind, t, lo, hi, float(x))[0]
            fd = richardson(lf, th[j], h)
            assert abs(d[j] - fd) <= 1e-7 * max(1.0, abs(fd)), (x, j, d[j], fd)


def test_argus_p_derivative_is_log_tau():
    # d log f / dp = log tau at fixed x (p appears only as the exponent)
    x, m0 = 5.25, 5.29
    lf = lambda p: oracle.leaf_logf("argus", [m0, -20.0, p], 5.2, 5.29, x)[0]
    _, d, _ = oracle.leaf_logf("argus", [m0, -20.0, 0.5], 5.2, 5.29, x)
    assert abs(d[2] - richardson(lf, 0.5, 1e-4)) < 1e-9


def test_argus_p_domain():
    for p in (0.0, -0.3):
        _, _, rc = oracle.leaf_norm("argus", [5.29, -20.0, p], 5.2, 5.29)
        assert rc == oracle.EDOMAIN


@pytest.mark.parametrize("m0,c,lo,hi", [(1.0, -3.0, 0.0, 1.5), (5.29, -20.0, 5.2, 5.29),
                                        (1.0, 4.0, 0.2, 0.9), (2.0, -0.7, 0.5, 1.9)])
def test_argus_p1_closed_form(m0, c, lo, hi):
    """p = 1: int tau e^{c tau} d tau = e^{c tau} (c tau - 1) / c^2, so
    I = (m0^2/2) [g(tau(lo)) - g(tau(b'))], b' = min(hi, m0)."""
    b = min(hi, m0)
    ta, tb = 1 - (lo / m0) ** 2, 1 - (b / m0) ** 2
    g = lambda t: math.exp(c * t) * (c * t - 1) / c**2
    want = 0.5 * m0 * m0 * (g(ta) - g(tb))
    I, dI, rc = oracle.leaf_norm("argus", [m0, c, 1.0], lo, hi)
    assert rc == 0 and abs(I - want) <= 1e-13 * want
    # d/dc of the closed form
    dg = lambda t: (math.exp(c * t) * (t * (c * t - 1) + t) * c**2 - 2 * c * math.exp(c * t) * (c * t - 1)) / c**4
    assert abs(dI[1] - 0.5 * m0 * m0 * (dg(ta) - dg(tb))) <= 1e-12 * abs(dI[1])


def test_argus_general_p_continuous_at_one_half():
    """The closed form at p = 1/2 and the quadrature just beside it agree."""
    th = [5.29, -20.0, 0.5]
    I, dI, _ = oracle.leaf_norm("argus", th, 5.2, 5.29)
    for e in (1e-9, -1e-9):
        Ie, dIe, rc = oracle.leaf_norm("argus", [5.29, -20.0, 0.5 + e], 5.2, 5.29)
        assert rc == 0
        assert abs(Ie - (I + e * dI[2])) <= 3e-13 * I + 1e-6 * abs(e * dI[2])
        np.testing.assert_allclose(dIe[:2], dI[:2], rtol=1e-7)


# ---------------------------------------------------------------- whole NLLs

def test_gaussian_nll_closed_form():
    """NLL = n log(sigma sqrt(2 pi) Z) + [S_xx + n (xbar-mu)^2]/(2 sigma^2)."""
    w = datagen.c1()
    x = w["cols"][0]
    mu, s = w["spec"]["params"]
    n, xb = len(x), x.mean()
    mp.mp.dps = 40
    Z = (mp.erf((10 - mu) / (mp.sqrt(2) * s)) - mp.erf((-10 - mu) / (mp.sqrt(2) * s))) / 2
    sxx = float(np.sum((x - xb) ** 2))
    want = n * float(mp.log(s * mp.sqrt(2 * mp.pi) * Z)) + (sxx + n * (xb - mu) ** 2) / (2 * s * s)
    got, g, rc = oracle.nll(w["spec"], w["spec"]["params"], w["cols"])
    assert rc == 0
    assert abs(got - want) <= 1e-13 * abs(want)
    # gradient closed form (Z = 1 to far below 1e-16 here)
    gmu = -n * (xb - mu) / s**2
    gs = n / s - (sxx + n * (xb - mu) ** 2) / s**3
    assert abs(g[0] - gmu) < 1e-9 * n and abs(g[1] - gs) < 1e-9 * n


def test_gaussian_ml_estimates_are_sample_moments():
    w = datagen.c1()
    x = w["cols"][0]
    xb = x.mean()
    sd = math.sqrt(np.mean((x - xb) ** 2))     # 1/n, not 1/(n-1)
    spec = dict(w["spec"])
    _, g, sc, rc = oracle.nll_scaled(spec, [xb, sd], w["cols"])
    assert rc == 0
    assert np.all(np.abs(g) <= 1e-10 * sc)
    # and the 1/(n-1) estimate is NOT a stationary point
    sd1 = math.sqrt(np.sum((x - xb) ** 2) / (len(x) - 1))
    _, g1, sc1, _ = oracle.nll_scaled(spec, [xb, sd1], w["cols"])
    assert abs(g1[1]) > 1e-6 * sc1[1]


EVENTS = np.array([0.3, 1.7, 4.9, 5.2, 9.1])


def test_add_fractions_hand_expanded():
    spec = datagen.gauss_exp_spec()
    mu, s, lam, f = 4.8, 0.7, -0.25, 0.3
    p = [mu, s, lam, f]
    pg = np.exp(lib_logpdf("gauss", [mu, s], 0, 10, EVENTS))
    pe = np.exp(lib_logpdf("exp", [lam], 0, 10, EVENTS))
    want = -np.sum(np.log(f * pg + (1 - f) * pe))
    got, g, rc = oracle.nll(spec, p, EVENTS)
    assert rc == 0 and abs(got - want) < 1e-12 * abs(want)
    # d/df = -sum (pg - pe)/P
    assert abs(g[3] + np.sum((pg - pe) / (f * pg + (1 - f) * pe))) < 1e-11
    lp, rc = oracle.logp(spec, p, EVENTS)
    np.testing.assert_allclose(lp, np.log(f * pg + (1 - f) * pe), rtol=0, atol=1e-12)


def test_three_component_add_fractions():
    spec = {"obs": [(0.0, 10.0)], "params": [5.0, 0.5, -0.3, 0.2, 0.3, 2.0, 1.0],
            "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]},
                      {"type": "exp", "obs": 0, "params": [2]},
                      {"type": "gauss", "obs": 0, "params": [5, 6]},
                      {"type": "add_frac", "children": [0, 2, 1], "params": [3, 4]}],
            "root": 3}
    p = spec["params"]
    g1 = np.exp(lib_logpdf("gauss", [5.0, 0.5], 0, 10, EVENTS))
    g2 = np.exp(lib_logpdf("gauss", [2.0, 1.0], 0, 10, EVENTS))
    e = np.exp(lib_logpdf("exp", [-0.3], 0, 10, EVENTS))
    want = -np.sum(np.log(0.2 * g1 + 0.3 * g2 + 0.5 * e))
    got, _, rc = oracle.nll(spec, p, EVENTS)
    assert rc == 0 and abs(got - want) < 1e-12 * abs(want)


def test_prod_is_sum_of_leaf_nlls():
    w = datagen.c3(n=3000, extended=False)
    spec, cols = w["spec"], w["cols"].astype(np.float64)
    p = spec["params"]
    got, g, rc = oracle.nll(spec, p, cols)
    assert rc == 0
    parts = 0.0
    for k, (kind, idx, (lo, hi)) in enumerate([("gauss", [0, 1], (-8, 8)),
                                                ("exp", [2], (0, 10)),
                                                ("cheb", [3, 4, 5, 6], (-1, 1))]):
        th = [p[i] for i in idx]
        parts -= np.sum(lib_logpdf(kind, th, lo, hi, cols[k]))
    assert abs(got - parts) < 1e-11 * abs(parts)


def test_extended_nll_and_yield_identity():
    spec = datagen.gauss_exp_ext_spec(nu_s=3.0, nu_b=4.5)
    p = [4.8, 0.7, -0.25, 3.0, 4.5]
    pg = np.exp(lib_logpdf("gauss", [4.8, 0.7], 0, 10, EVENTS))
    pe = np.exp(lib_logpdf("exp", [-0.25], 0, 10, EVENTS))
    want = 7.5 - np.sum(np.log(3.0 * pg + 4.5 * pe))
    got, g, rc = oracle.nll(spec, p, EVENTS)
    assert rc == 0 and abs(got - want) < 1e-12 * abs(want)
    # sum_k nu_k dNLL/dnu_k = sum nu - n at every point
    assert abs(p[3] * g[3] + p[4] * g[4] - (7.5 - len(EVENTS))) < 1e-12


def test_extended_mle_yields_sum_to_n():
    w = datagen.c4(toys=1, nu_s_range=(800, 800.0001), nu_b_range=(2000, 2000.0001))
    spec, cols = w["spec"], w["cols"]
    n = cols.shape[1]
    shape = [5.0, 0.5, -0.3]
    nu = np.array([700.0, 2100.0])
    for _ in range(60):  # Newton on the yields with the shape held fixed
        _, g, _ = oracle.nll(spec, [*shape, *nu], cols)
        h = 1e-3
        H = np.zeros((2, 2))
        for j in range(2):
            d = np.zeros(2)
            d[j] = h
            gp = oracle.nll(spec, [*shape, *(nu + d)], cols)[1][3:]
            gm = oracle.nll(spec, [*shape, *(nu - d)], cols)[1][3:]
            H[:, j] = (gp - gm) / (2 * h)
        nu = nu - np.linalg.solve(H, g[3:])
    assert abs(nu.sum() - n) < 1e-8 * n


def test_crystal_ball_continuity_at_junction():
    m0, s, a, n = 0.0, 1.0, 1.3, 2.7
    th = [m0, s, a, n]
    xj = m0 - a * s
    for eps in (1e-9, 1e-11):
        lo_side = oracle.leaf_logf("cb", th, -5, 5, xj - eps)
        hi_side = oracle.leaf_logf("cb", th, -5, 5, xj + eps)
        assert abs(lo_side[0] - hi_side[0]) < 10 * eps
        # d log f / d m0 = slope in t times -1/sigma: continuous
        assert abs(lo_side[1][0] - hi_side[1][0]) < 1e-6
        assert abs(lo_side[1][2]) < 1e-6 and abs(hi_side[1][2]) == 0.0


def test_exponential_lambda_to_zero():
    """At lambda = 0 the integral is the range length; near 0 it follows the
    moments: I = int e^{lx} ~ L + l M1 + l^2 M2/2, dI/dl ~ M1 + l M2."""
    lo, hi = -2.0, 3.0
    M1, M2, M3 = (hi**2 - lo**2) / 2, (hi**3 - lo**3) / 3, (hi**4 - lo**4) / 4
    I0, d0, _ = oracle.leaf_norm("exp", [0.0], lo, hi)
    assert I0 == hi - lo
    assert abs(d0[0] - M1) < 1e-15
    for lam in (1e-9, -1e-9, 1e-6, -3e-4, 1e-3):
        I, d, _ = oracle.leaf_norm("exp", [lam], lo, hi)
        assert abs(I - (I0 + lam * M1 + lam**2 * M2 / 2)) < abs(lam) ** 3 * M3 + 1e-14
        assert abs(d[0] - (M1 + lam * M2 + lam**2 * M3 / 2)) < 10 * abs(lam) ** 3 * M3 + 1e-13


MODELS_FOR_FD = {
    "gauss_exp_frac": (datagen.gauss_exp_spec(), [5.1, 0.55, -0.27, 0.23],
                       lambda: datagen.c2(n=4000)["cols"]),
    "prod3_ext": (datagen.prod3_spec(2000.0), [0.1, 1.6, -0.45, 0.22, -0.08, 0.06, 0.03, 2100.0],
                  lambda: datagen.c3(n=2000)["cols"].astype(np.float64)),
    "cb_argus_ext": (datagen.cb_argus_spec(300.0, 3000.0),
                     [5.2793, 0.0032, 1.6, 3.2, 5.29, -19.0, 0.5, 320.0, 2950.0],
                     lambda: datagen.c5(300, 3000)["cols"].astype(np.float64),
                     [0.003, 0.003, 1.5, 3.0, 0.01, 20.0, 1.0, 300.0, 3000.0]),
    "cb_highside_frac": ({"obs": [(-6.0, 6.0)], "params": [0.1, 0.9, -1.1, 2.2, -0.2, 0.4],
                          "nodes": [{"type": "cb", "obs": 0, "params": [0, 1, 2, 3]},
                                    {"type": "exp", "obs": 0, "params": [4]},
                                    {"type": "add_frac", "children": [0, 1], "params": [5]}],
                          "root": 2}, [0.1, 0.9, -1.1, 2.2, -0.2, 0.4],
                         lambda: np.linspace(-5.9, 5.9, 777)),
}


@pytest.mark.parametrize("name", sorted(MODELS_FOR_FD))
def test_gradient_matches_richardson_differences(name):
    spec, p0, data, *scales = MODELS_FOR_FD[name]
    scales = scales[0] if scales else [max(abs(v), 1e-2) for v in p0]
    cols = data()
    _, g, sc, rc = oracle.nll_scaled(spec, p0, cols)
    assert rc == 0
    fixed = spec.get("fixed", [False] * len(p0))
    for j in range(len(p0)):
        if fixed[j]:
            continue
        h = 1e-4 * scales[j]

        def f(v):
            p = list(p0)
            p[j] = v
            return oracle.nll(spec, p, cols, grad=False)[0]
        fd = richardson(f, p0[j], h)
        assert abs(g[j] - fd) <= 1e-8 * sc[j], (j, g[j], fd, sc[j])


def test_result_independent_of_thread_count():
    w = datagen.c2(n=50_000)
    a = oracle.nll(w["spec"], w["spec"]["params"], w["cols"], nthreads=1)
    b = oracle.nll(w["spec"], w["spec"]["params"], w["cols"], nthreads=4)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_batched_equals_single_segments():
    w = datagen.c4(toys=5, nu_s_range=(50, 500), nu_b_range=(100, 1000))
    out, rc = oracle.nll_batched(w["spec"], w["cols"], w["offsets"], w["params_matrix"])
    assert rc == 0
    for t in range(5):
        b, e = w["offsets"][t], w["offsets"][t + 1]
        v, g, _ = oracle.nll(w["spec"], w["params_matrix"][t], w["cols"][:, b:e])
        assert out[t, 0] == v and np.array_equal(out[t, 1:], g)


def test_domain_errors_give_infinite_nll():
    spec = datagen.gauss_exp_spec()
    x = np.array([1.0, 2.0])
    assert oracle.nll(spec, [5.0, -0.5, -0.3, 0.2], x)[0] == math.inf
    assert oracle.nll(spec, [5.0, 0.5, -0.3, 1.2], x)[0] == math.inf
    cheb = {"obs": [(-1.0, 1.0)], "params": [1.5],
            "nodes": [{"type": "cheb", "obs": 0, "params": [0]}], "root": 0}
    v, _, rc = oracle.nll(cheb, [1.5], np.array([-0.9, 0.5]))   # 1 + 1.5 x < 0
    assert v == math.inf and rc == oracle.EDOMAIN
    bad_prod = {"obs": [(0.0, 1.0)], "params": [0.5, 1.0, -1.0],
                "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]},
                          {"type": "exp", "obs": 0, "params": [2]},
                          {"type": "prod", "children": [0, 1]}], "root": 2}
    assert oracle.nll(bad_prod, [0.5, 1.0, -1.0], x)[2] == oracle.EUNSUPPORTED


def test_adam_step_properties():
    """Adam (Kingma & Ba 2015): the bias-corrected first step has size lr in
    every coordinate (m_hat/sqrt(v_hat) = g/|g|), and a constant gradient keeps
    the step at lr; entries that are not free never move."""
    th = np.array([1.0, 2.0, 3.0])
    scale = np.array([1.0, 0.5, 2.0])
    m1, m2 = np.zeros(3), np.zeros(3)
    g = np.array([3.0, -0.2, 7.0])
    oracle.adam_step(th, g, scale, [1, 1, 0], m1, m2, 1, 0.01, eps=0.0)
    np.testing.assert_allclose(th, [1.0 - 0.01, 2.0 + 0.005, 3.0], rtol=0, atol=1e-15)
    for t in range(2, 6):
        before = th.copy()
        oracle.adam_step(th, g, scale, [1, 1, 0], m1, m2, t, 0.01, eps=0.0)
        np.testing.assert_allclose(before - th, [0.01, -0.005, 0.0], rtol=1e-12, atol=1e-15)
