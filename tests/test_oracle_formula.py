"""Pins of the oracle's formula leaves (type "formula"): a PDF given as text, as the
formula PDFs of Sec. 4 are, evaluated by walking its parse tree with forward
derivatives and normalised by adaptive Gauss-Legendre quadrature.

- Formulas that spell out a built-in leaf (Gaussian, Exponential, Chebychev,
  Johnson SU) give that leaf's log density, derivatives, integral and integral
  derivatives (the built-ins are pinned to scipy and quadrature in
  test_oracle_pins.py), and whole-model NLLs and gradients equal the built-in
  model's.
- Values agree with Python's own evaluation of the same text; derivatives
  with Richardson differences; integrals with mpmath quadrature and, for a
  Breit-Wigner, with its arctangent closed form.
- Precedence, associativity, integer powers of negative bases, and rejected
  syntax."""
import math

import mpmath as mp
import numpy as np
import pytest
import scipy.special as sps

import datagen
import oracle

GAUSS = "exp(-0.5*((x-p0)/p1)^2)"
JOHNSON = ("p3/(p1*2.5066282746310002)*exp(-0.5*(p2+p3*asinh((x-p0)/p1))^2)"
           "/sqrt(1+((x-p0)/p1)^2)")   # 2.50662... = sqrt(2 pi)
CHEB = "1 + p0*u + p1*(2*u^2-1) + p2*(4*u^3-3*u) + p3*(8*u^4-8*u^2+1)"


def cheb_text(lo, hi):
    u = f"((2*x-({lo})-({hi}))/(({hi})-({lo})))"
    return CHEB.replace("u", u)


BUILTIN = [
    ("gauss", GAUSS, [0.25, 1.1], -10.0, 10.0),
    ("gauss", GAUSS, [5.0, 0.5], 0.0, 10.0),
    ("exp", "exp(p0*x)", [-0.3], 0.0, 10.0),
    ("exp", "exp(p0*x)", [0.7], -1.0, 2.0),
    ("cheb", None, [0.2, -0.1, 0.05, 0.02], -1.0, 1.0),
    ("cheb", None, [0.3, 0.1, -0.05, 0.01], 2.0, 7.0),
    ("johnson", JOHNSON, [0.5, 1.3, -0.4, 1.7], -2.0, 3.0),
]


@pytest.mark.parametrize("kind,text,th,lo,hi", BUILTIN)
def test_formula_equals_builtin_leaf(kind, text, th, lo, hi):
    text = text or cheb_text(lo, hi)
    I, dI, rc = oracle.expr_norm(text, th, lo, hi)
    Ib, dIb, rcb = oracle.leaf_norm(kind, th, lo, hi)
    assert rc == rcb == 0
    assert abs(I - Ib) <= 1e-13 * Ib
    scale = 1e-13 * max(Ib, np.max(np.abs(dIb)))
    np.testing.assert_allclose(dI, dIb, rtol=0, atol=scale)
    for x in np.linspace(lo, hi, 13):
        lf, d, rc = oracle.expr_logf(text, th, float(x))
        lfb, db, _ = oracle.leaf_logf(kind, th, lo, hi, float(x))
        assert rc == 0 and abs(lf - lfb) <= 1e-13 * max(1.0, abs(lfb))
        np.testing.assert_allclose(d, db, rtol=1e-12, atol=1e-12)


def np_eval(text, th, x):
    env = {"exp": np.exp, "log": np.log, "sqrt": np.sqrt, "sin": np.sin, "cos": np.cos,
           "tanh": np.tanh, "sinh": np.sinh, "cosh": np.cosh, "asinh": np.arcsinh,
           "atan": np.arctan, "erf": sps.erf, "erfc": sps.erfc, "abs": np.abs,
           "pow": np.power, "x": x}
    env.update({f"p{j}": v for j, v in enumerate(th)})
    return eval(text.replace("^", "**"), {"__builtins__": {}}, env)


FORMULAS = [
    ("1/(1+((x-p0)/p1)^2)", [0.4, 0.7], -3.0, 4.0),                    # Breit-Wigner
    ("x^2*exp(-p0*x) + p1", [1.3, 0.05], 0.0, 8.0),
    ("(1 + p0*sin(3*x))*exp(-abs(x)/p1)", [0.3, 2.0], -4.0, 5.0),      # kink at 0
    ("erfc((x-p0)/p1) + 0.2*tanh(x) + 1", [1.0, 0.6], -2.0, 6.0),
    ("sqrt(1+x^2)*cosh(p0*x)/(2+sinh(p1*x)^2) + atan(x)^2", [0.3, 0.5], -3.0, 3.0),
    ("pow(x, p0)*exp(-x/p1)", [1.7, 1.5], 0.1, 9.0),                    # non-integer power
    ("exp(-x*p0) * log(2+x) * erf(x+3) + 1e-3", [0.8], -1.0, 5.0),
]


@pytest.mark.parametrize("text,th,lo,hi", FORMULAS)
def test_values_match_python_and_derivatives_match_differences(text, th, lo, hi):
    assert oracle.expr_check(text, len(th)) == 0
    for x in np.linspace(lo, hi, 11)[1:-1] + 0.013:
        lf, d, rc = oracle.expr_logf(text, th, float(x))
        assert rc == 0
        want = math.log(np_eval(text, th, x))
        assert abs(lf - want) <= 1e-14 * max(1.0, abs(want))
        for j in range(len(th)):
            h = 1e-4 * max(abs(th[j]), 0.1)

            def g(v):
                t = list(th)
                t[j] = v
                return math.log(np_eval(text, t, x))
            fd = (4 * (g(th[j] + h / 2) - g(th[j] - h / 2)) / h - (g(th[j] + h) - g(th[j] - h)) / (2 * h)) / 3
            assert abs(d[j] - fd) <= 1e-8 * max(1.0, abs(fd)), (x, j, d[j], fd)


@pytest.mark.parametrize("text,th,lo,hi", FORMULAS)
def test_integral_matches_quadrature(text, th, lo, hi):
    mp.mp.dps = 30
    I, dI, rc = oracle.expr_norm(text, th, lo, hi)
    assert rc == 0
    f = lambda x: np_eval(text.replace("abs", "fabs"), th, x)
    env_text = text
    pts = [lo, 0.0, hi] if lo < 0.0 < hi else [lo, hi]

    def fm(x):
        e = {"exp": mp.exp, "log": mp.log, "sqrt": mp.sqrt, "sin": mp.sin, "cos": mp.cos,
             "tanh": mp.tanh, "sinh": mp.sinh, "cosh": mp.cosh, "asinh": mp.asinh,
             "atan": mp.atan, "erf": mp.erf, "erfc": mp.erfc, "abs": abs, "pow": mp.power,
             "x": x}
        e.update({f"p{j}": mp.mpf(v) for j, v in enumerate(th)})
        return eval(env_text.replace("^", "**"), {"__builtins__": {}}, e)
    want = float(mp.quad(fm, pts))
    assert abs(I - want) <= 1e-13 * abs(want), (I, want)
    del f
    # derivatives of the integral against Richardson differences of it
    for j in range(len(th)):
        h = 1e-3 * max(abs(th[j]), 0.1)

        def Ij(v):
            t = list(th)
            t[j] = v
            return oracle.expr_norm(text, t, lo, hi)[0]
        fd = (4 * (Ij(th[j] + h / 2) - Ij(th[j] - h / 2)) / h - (Ij(th[j] + h) - Ij(th[j] - h)) / (2 * h)) / 3
        assert abs(dI[j] - fd) <= 1e-8 * max(abs(fd), 1e-3 * I), (j, dI[j], fd)


def test_breit_wigner_integral_closed_form():
    for m, g, lo, hi in [(0.4, 0.7, -3.0, 4.0), (91.19, 2.5, 60.0, 120.0), (0.0, 0.01, -1.0, 1.0)]:
        I, dI, rc = oracle.expr_norm("1/(1+((x-p0)/p1)^2)", [m, g], lo, hi)
        want = g * (math.atan((hi - m) / g) - math.atan((lo - m) / g))
        assert rc == 0 and abs(I - want) <= 1e-13 * want, (m, g, I, want)
        # dI/dm = 1/(1+((lo-m)/g)^2) - 1/(1+((hi-m)/g)^2)
        dm = 1 / (1 + ((lo - m) / g) ** 2) - 1 / (1 + ((hi - m) / g) ** 2)
        assert abs(dI[0] - dm) <= 1e-12 * max(1.0, abs(dm))


@pytest.mark.parametrize("text,value", [
    ("2^3^2", 512.0),            # right-associative
    ("-2^2+5", 1.0),             # unary minus below '^'
    ("(-2)^2", 4.0),
    ("2*3+4", 10.0), ("2+3*4", 14.0), ("10/2/5", 1.0), ("8-2-3", 3.0),
    ("2^-1", 0.5), ("pow(-2, 3) + 9", 1.0), ("(-1.5)^2", 2.25),
    ("1e-3*1000", 1.0), (".5*4", 2.0), ("2.5E+1/25", 1.0), ("+3", 3.0),
    ("exp(0)+log(1)+sqrt(4)+abs(-1)", 4.0), ("--2", 2.0),
])
def test_precedence_and_literals(text, value):
    lf, _, rc = oracle.expr_logf(text, [], 0.0)
    assert rc == 0 and abs(lf - math.log(value)) < 1e-15


@pytest.mark.parametrize("text,npar", [
    ("", 0), ("1+", 0), ("x)", 0), ("(x", 0), ("p2", 2), ("foo(x)", 0), ("exp x", 0),
    ("1e", 0), ("x x", 0), ("pow(x)", 0), ("exp(x,1)", 0), ("p", 1), ("y", 0), ("1..2", 0),
    ("x^", 0), ("*x", 0),
])
def test_rejected_syntax(text, npar):
    assert oracle.expr_check(text, npar) == oracle.EINVAL


def test_model_with_formula_leaf_equals_builtin_model():
    spec = datagen.gauss_exp_ext_spec(nu_s=300.0, nu_b=700.0)
    cols = datagen.c4(toys=1)["cols"][:, :1000]
    alt = {**spec, "nodes": [dict(spec["nodes"][0], type="formula", formula=GAUSS),
                             dict(spec["nodes"][1], type="formula", formula="exp(p0*x)"),
                             spec["nodes"][2]]}
    p = [5.05, 0.52, -0.28, 310.0, 690.0]
    v, g, rc = oracle.nll(spec, p, cols)
    va, ga, rca = oracle.nll(alt, p, cols)
    assert rc == rca == 0
    assert abs(va - v) <= 1e-13 * abs(v)
    np.testing.assert_allclose(ga, g, rtol=1e-11, atol=1e-9)
    lp, _ = oracle.logp(spec, p, cols)
    lpa, _ = oracle.logp(alt, p, cols)
    np.testing.assert_allclose(lpa, lp, rtol=0, atol=1e-13)


def test_formula_domain_and_generation():
    spec = {"obs": [(-1.0, 1.0)], "params": [0.5],
            "nodes": [{"type": "formula", "formula": "x - p0", "obs": 0, "params": [0]}], "root": 0}
    v, g, rc = oracle.nll(spec, [0.5], np.array([[0.7, 0.9]]))
    assert rc == oracle.EDOMAIN and v == math.inf          # integral <= 0
    bad = {**spec, "nodes": [dict(spec["nodes"][0], formula="x +")]}
    assert oracle.nll(bad, [0.5], np.array([[0.7]]))[2] == oracle.EINVAL
    ok = {**spec, "nodes": [dict(spec["nodes"][0], formula="1 + p0*x")]}
    assert oracle.generate(ok, [[0.5]], [[3]], [0, 3], seed=1, col_f32=False)[2] == oracle.EUNSUPPORTED
