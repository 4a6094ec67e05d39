"""Shared helpers for the parity tests: error metrics and tolerances.

Tolerances (relative NLL error; gradient error in the L1 metric
|g - g_ref|_k / sum_i |d ell_i / d theta_k|, because the gradient itself goes
to zero at the minimum):
  FP64 evaluation   NLL <= 1e-12, gradient <= 1e-10
  FP32 evaluation   NLL <= 1e-7,  gradient <= 1e-6
FP32 evaluation rounds each event's log-density at ~6e-8 relative; each
thread's sums are Kahan-compensated in FP32, a block adds them in FP32 pairs
(about 48 significant bits) and converts its totals to FP64 once, and every
sum above the block is FP64, so the NLL error stays near the per-event
rounding (1e-7 allows one unit of the last place in the worst event to be
systematic); the gradient bound is the target the method is held to.
Per-event log P: FP64 within 2e-14 * max(1, |log P|) (the batch-vs-classic
accuracy of the paper's Sec. 5.3 on log-likelihoods), FP32 within
2e-6 * max(1, |log P|).
"""
import math

import numpy as np

TOL = {"fp64": {"nll": 1e-12, "grad": 1e-10, "logp": 2e-14},
       "fp32": {"nll": 1e-7, "grad": 1e-6, "logp": 2e-6}}


def rel_nll(got, want):
    return abs(got - want) / max(abs(want), 1e-300)


def grad_l1(got, want, scale, free):
    g = np.asarray(got, np.float64)
    w = np.asarray(want, np.float64)
    s = np.asarray(scale, np.float64)
    err = np.zeros_like(g)
    for k in range(len(g)):
        if not free[k]:
            continue
        err[k] = abs(g[k] - w[k]) / max(s[k], 1e-300)
    return err


def free_mask(spec):
    fx = spec.get("fixed") or [False] * len(spec["params"])
    return [not f for f in fx]


def logp_err(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    return np.abs(got - want) / np.maximum(1.0, np.abs(want))


def dtype_of(w):
    return w["dtype"]


def finite(x):
    return x is not None and math.isfinite(x)
