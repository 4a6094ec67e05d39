#!/usr/bin/env python3
"""Benchmark: fused unbinned NLL + adjoint gradient on one GB300 (or N, as
independent weak-scaling replicas launched by torchrun).

A step is one pass of the hot path over one batch: the FP64 prologue
(normalisation integrals, coefficients), the per-event log-density and adjoint
of every event, the compensated reduction and the FP64 epilogue -- one fused
kernel launch through the C-ABI (rf_nll).

Default workload: the B-factory-shaped mass fit -- Crystal Ball (5.279, 0.003,
1.5, 3) + ARGUS (5.29, -20, 1/2), extended yields 1e6 + 1e8, 1.01e8 events in
one FP32 column, 7 free parameters; FP32 per-event arithmetic with FP64
normalisation, reduction and gradient accumulation.  The event column (404 MB)
is larger than L2 (129 MB), so no flush is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the reference implementation the GPU results are checked against) on the
host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NLL+grad events/s on 1 GB300 (fused vs plain FP64), % roofline; toy NLLs/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    d = dict(FALLBACK_PEAKS)
    d["source"] = "fallback"
    return d


L2_BYTES = 129 << 20


class L2Flush:
    """Empties L2 between timed calls: writes a buffer twice the L2, then reads
    another one of that size, so that the write-backs of the written lines
    happen here (outside the timed region) and L2 is left holding clean lines
    of the read buffer; a timed call then pays for its own traffic only."""

    def __init__(self, torch, nbytes=2 * L2_BYTES):
        self.w = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.zero_()
        return self.r.sum()


def make_workload(name):
    import datagen
    if name == "c5":
        return datagen.c5()
    if name == "c3":
        return datagen.c3()
    if name == "c2":
        return datagen.c2()
    if name == "c1":
        return datagen.c1()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.tmp = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.tmp.close()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def cpu_oracle_rate(w, sample_events, nthreads=0):
    """Oracle events/s (NLL + analytic gradient, FP64) on the first
    `sample_events` events of the workload, all allowed host cores."""
    import numpy as np

    import oracle
    cols = np.ascontiguousarray(w["cols"][:, :sample_events].astype(np.float64))
    p = w["spec"]["params"]
    oracle.nll(w["spec"], p, cols[:, :1000], nthreads=nthreads)  # load / warm
    t0 = time.perf_counter()
    v, g, rc = oracle.nll(w["spec"], p, cols, nthreads=nthreads)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if nthreads <= 0 else nthreads
    return cols.shape[1] / dt, cores, dt


# FP32-pipe instructions per event of the fused kernel's formulation, by piece
# (derived op by op from the formulas of each leaf, the log of the mixture and
# the adjoint sums; the secondary "issue" figure of the bench line).
# leaf type -> (base, extra per wanted derivative by leaf-parameter index,
#               shared extra when any derivative is wanted)
# Per-event logarithms are taken in base 2 (one hardware lg2 each, no
# conversion factor); a location shift is one subtraction and one FMA; each
# component's log-coefficient is folded into its first leaf (no addition);
# the two-term log-sum-exp is one ex2, one lg2 and one reciprocal with the
# arithmetic around them.
LEAF_INSTR = {
    "gauss": (4, {0: 0, 1: 0}, 0),
    "exp": (3, {0: 0}, 0),                  # 1 when the range starts at 0 (no shift)
    "cheb": (11, {0: 1, 1: 1, 2: 1, 3: 1}, 1),
    "cb": (8, {0: 0, 1: 1, 2: 3, 3: 3}, 3),
    # p = 1/2 on m0^2 - x^2 (no normalising multiply); d/dm0 needs tau (+1 of
    # its 7); a free p: the general form (+3) and d/dp (+2)
    "argus": (9, {0: 7, 1: 0, 2: 5}, 0),
    "johnson": (12, {0: 0, 1: 1, 2: 0, 3: 1}, 5),
}
F64_TO_F32_INSTR = 9   # integer-pipe rounding of an FP64 column value


# The compensated sums are counted at the largest chunk the kernels take (16
# events), so that the count is a property of the computation, not of the
# launch configuration that the tuner picks.
REF_EPT = 16


def algorithmic_instr_per_event(spec: dict, ept: int = REF_EPT, f64_columns: bool = False) -> float:
    nodes = spec["nodes"]
    fixed = spec.get("fixed") or [False] * len(spec["params"])
    leaves = [nd for nd in nodes if nd["type"] in LEAF_INSTR]
    root = nodes[spec.get("root", len(nodes) - 1)]
    nc = len(root["children"]) if root["type"] in ("add_frac", "add_ext") else 1
    total, free = 0.0, 0
    for lf in leaves:
        base, per, shared = LEAF_INSTR[lf["type"]]
        if lf["type"] == "exp" and spec["obs"][lf["obs"]][0] == 0.0:
            base = 1
        wanted = [j for j, p in enumerate(lf["params"]) if not fixed[p] and j in per]
        total += base + (shared if wanted else 0) + sum(per[j] for j in wanted)
        free += len(wanted)
    total += len(leaves) - nc                 # sums of a component's leaves
    if nc == 2:
        total += 11                           # two-term log-sum-exp and weights
    elif nc > 2:
        total += 11 * nc + 24
    total += 1 + (nc if nc > 1 else 1) + free  # adjoint sums
    total += 4.0 * (1 + nc + free) / ept      # compensated per-iteration sums
    total += 1                                # loads and loop
    if f64_columns:
        total += F64_TO_F32_INSTR * len(spec["obs"])
    return total


# The roofline of a step: t_roof = max(n B / BW, n sum_op N_op / R_op).  N_op
# are the minimal operation counts per event of each workload's formulas (the
# leaf densities, the log of the mixture, the adjoint sums), B the bytes a step
# must read per event, BW the measured HBM copy bandwidth, and R_op the
# throughput of each operation measured alone on this GPU by rf_microbench --
# for FP32 evaluation the hardware approximations the kernels issue (base-2
# exp and log, reciprocal, square root: the fastest form of each, so the
# roofline is the strict one), for FP64 evaluation the FP64 functions the
# kernels call (exp2, log2, division, sqrt) and the FP64 FMA.
OPS_PER_EVENT = {
    "c1": {"fma": 6},                                          # 3 FMA + 3 sums
    "c2": {"exp": 2, "log": 1, "rcp": 1, "fma": 6},
    "c3": {"log": 1, "rcp": 1, "fma": 16},                     # Clenshaw(4) 8 + 8 sums
    "c4": {"exp": 2, "log": 1, "rcp": 1, "fma": 6},
    "c5": {"exp": 2, "log": 2, "sqrt": 1, "rcp": 1, "fma": 8},
}
RATE_KEYS = {
    "fp32": {"exp": "ex2_approx_f32", "log": "lg2_approx_f32", "rcp": "rcp_approx_f32",
             "sqrt": "sqrt_approx_f32", "fma": "fp32_fma"},
    "fp64": {"exp": "exp2_f64", "log": "log2_f64", "rcp": "div_f64", "sqrt": "sqrt_f64",
             "fma": "fp64_fma"},
}


def roofline_8d(cfg: str, prec: str, n: int, bytes_per_event: float, step_ms: float,
                rates: dict, hbm_gbs: float) -> dict:
    """The fraction of the roofline reached by a step of `n` events that took
    step_ms: t_roof / t_step, with t_roof from the op list above."""
    ops = OPS_PER_EVENT[cfg]
    t_ops = {k: n * v / rates[RATE_KEYS[prec][k]] for k, v in ops.items()}
    t_compute = sum(t_ops.values())
    t_hbm = n * bytes_per_event / (hbm_gbs * 1e9)
    t_roof = max(t_compute, t_hbm)
    t = step_ms * 1e-3
    return {"bound": "alu" if t_compute >= t_hbm else "hbm", "unit": "events/s",
            "achieved": n / t, "peak": n / t_roof, "frac": t_roof / t,
            "t_roof_us": t_roof * 1e6, "t_compute_us": t_compute * 1e6, "t_hbm_us": t_hbm * 1e6,
            "step_us": t * 1e6, "ops_per_event": ops,
            "op_us": {k: v * 1e6 for k, v in t_ops.items()},
            "bytes_per_event": bytes_per_event,
            "rates": {RATE_KEYS[prec][k]: rates[RATE_KEYS[prec][k]] for k in ops}}


def profiled_traffic(kernel_hash: str):
    """DRAM bytes per launch from a committed ncu summary taken on exactly this
    kernel (matched by its source hash), else None."""
    import glob
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        # one (kernel_hash, dram_bytes_per_launch) pair per kernel section
        cur = None
        with open(path) as f:
            for line in f:
                key, _, val = line.partition("=")
                key, val = key.strip(), val.strip().strip("`")
                if key == "kernel_hash":
                    cur = val
                elif key == "dram_bytes_per_launch" and cur == kernel_hash and cur != "n/a":
                    return float(val)
    return None


def max_over_ranks(x: float, dist, device: str) -> float:
    """The slowest rank's value (every rank gets it); x itself on one rank."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(events_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job events/s: every rank (an independent replica on its own GPU)
    processes events_per_rank per step; the step time is the slowest rank's."""
    return world * events_per_rank / (ms_per_step * 1e-3)


def toy_study(rf, torch, toys=4096, iters=50, rates=None, hbm_gbs=None):
    """Toy NLLs/s: 4096 extended Gauss+Exp toys (about 1.3e8 FP64 events), one
    batched evaluation and a 50-iteration Adam fit replayed from a CUDA graph,
    FP32 and FP64 per-event arithmetic."""
    import numpy as np

    import datagen
    w = datagen.c4(toys=toys)
    ev = torch.from_numpy(w["cols"]).cuda()
    off = torch.from_numpy(w["offsets"]).cuda()
    res = {"toys": toys, "events": int(w["offsets"][-1]), "iters": iters}
    for prec in ("fp32", "fp64"):
        G = rf.Graph(w["spec"], "f64", prec)
        G.bind_events(ev, toys)
        pm = torch.from_numpy(w["params_matrix"]).cuda()
        G.nll_batched(off, pm)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            G.nll_batched(off, pm)
        b.record()
        torch.cuda.synchronize()
        t_eval = a.elapsed_time(b) / 5
        scale = torch.from_numpy(np.maximum(np.abs(w["params_matrix"]), 1.0)).cuda()
        t0 = time.perf_counter()
        G.fit_toys(off, pm, scale, iters, 1e-2)
        t_fit = (time.perf_counter() - t0) * 1e3
        res[prec] = {"eval_ms": t_eval, "toy_nll_per_s": toys / (t_eval * 1e-3),
                     "events_per_s": res["events"] / (t_eval * 1e-3),
                     "fit_ms": t_fit, "fit_toy_iters_per_s": toys * iters / (t_fit * 1e-3),
                     "launches_per_fit": G.last_launches(), "kernel": G.uses_jit()}
        if rates:
            # FP32 evaluation reads the FP32 copy of the columns made once at bind
            res[prec]["roofline"] = roofline_8d("c4", prec, res["events"],
                                                4 if prec == "fp32" else 8, t_eval, rates,
                                                hbm_gbs)
    # toy generation on the device: the same 4096 toys (per-component counts
    # = the workload's signal / background split), FP64 columns
    G = rf.Graph(w["spec"], "f64", "fp64")
    counts = torch.from_numpy(np.rint(w["params_matrix"][:, 3:5]).astype(np.int64)).cuda()
    goff = torch.zeros(toys + 1, dtype=torch.int64, device="cuda")
    goff[1:] = torch.cumsum(counts.sum(1), 0)
    pmg = torch.from_numpy(w["params_matrix"]).cuda()
    ng = int(goff[-1].item())
    buf = torch.empty(1, ng, dtype=torch.float64, device="cuda")
    G.generate_toys(pmg, counts, goff, seed=1, out=buf)
    torch.cuda.synchronize()
    a.record()
    for _ in range(3):
        G.generate_toys(pmg, counts, goff, seed=2, out=buf)
    b.record()
    torch.cuda.synchronize()
    t_gen = a.elapsed_time(b) / 3
    res["generation"] = {"events": ng, "ms": t_gen, "events_per_s": ng / (t_gen * 1e-3),
                         "toys_per_s": toys / (t_gen * 1e-3)}
    return res


def small_configs(rf, torch, rates=None, hbm_gbs=None):
    """Per-call latency of the small workloads (C1 1e4, C2 1e6, C3 1e7 events):
    a host loop of calls on one stream, and the same calls replayed from a
    CUDA graph (GPU time only); C2 (8 MB) and C3 (120 MB) also with L2
    flushed before every call (L2Flush).  FP32 evaluation, plus FP64
    evaluation for C1 and C2; C2 and C3 at the tuner's launch."""
    import numpy as np

    res = {}
    flush = L2Flush(torch)
    for name, precs in (("c1", ("fp64", "fp32")), ("c2", ("fp64", "fp32")), ("c3", ("fp32",))):
        w = make_workload(name)
        ev = torch.from_numpy(np.ascontiguousarray(w["cols"])).cuda()
        n = w["cols"].shape[1]
        params = torch.tensor(w["spec"]["params"], dtype=torch.float64, device="cuda")
        for prec in precs:
            G = rf.Graph(w["spec"], w["dtype"], prec)
            if name in ("c2", "c3"):  # events enough for the launch shape to matter
                G.tune(ev, params)
            out = torch.empty(1 + len(w["spec"]["params"]), dtype=torch.float64, device="cuda")
            for _ in range(20):
                G.nll(ev, params, out=out)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = 200
            a.record()
            for _ in range(k):
                G.nll(ev, params, out=out)
            b.record()
            torch.cuda.synchronize()
            r = {"events": n, "stream_us": a.elapsed_time(b) * 1e3 / k,
                 "launch": G.get_launch()}
            try:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    for _ in range(20):
                        G.nll(ev, params, out=out)
                g.replay()
                torch.cuda.synchronize()
                a.record()
                for _ in range(10):
                    g.replay()
                b.record()
                torch.cuda.synchronize()
                r["graph_us"] = a.elapsed_time(b) * 1e3 / 200
            except Exception as exc:  # capture unsupported here: report why
                r["graph_us"] = None
                r["graph_error"] = str(exc)[:200]
            if name in ("c2", "c3"):
                ts = []
                for _ in range(20):
                    flush()
                    a.record()
                    G.nll(ev, params, out=out)
                    b.record()
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b) * 1e3)
                r["cold_us_median"] = statistics.median(ts)
            r["events_per_s_graph"] = n / (r["graph_us"] * 1e-6) if r.get("graph_us") else None
            if rates and r.get("graph_us"):
                bpe = w["cols"].shape[0] * (4 if w["dtype"] == "f32" else 8)
                r["roofline"] = roofline_8d(name, prec, n, bpe, r["graph_us"] * 1e-3, rates,
                                            hbm_gbs)
                if "cold_us_median" in r:
                    r["roofline_cold"] = roofline_8d(name, prec, n, bpe,
                                                     r["cold_us_median"] * 1e-3, rates, hbm_gbs)
            res[f"{name}_{prec}"] = r
    res["c3_fp32_n_odd"] = odd_length_c3(rf, torch, rates, hbm_gbs)
    res["formula_leaves"] = formula_vs_builtin(rf, torch)
    return res


def odd_length_c3(rf, torch, rates=None, hbm_gbs=None):
    """C3 with 10,000,001 events: the three FP32 columns start at different
    16-byte phases (column j at j * n * 4 bytes), so the fused kernel reads
    them with 32-bit loads; per-event time against the 10,000,000-event run."""
    import numpy as np

    import datagen
    w = datagen.c3(n=10_000_001)
    ev = torch.from_numpy(np.ascontiguousarray(w["cols"])).cuda()
    n = w["cols"].shape[1]
    params = torch.tensor(w["spec"]["params"], dtype=torch.float64, device="cuda")
    G = rf.Graph(w["spec"], w["dtype"], "fp32")
    G.tune(ev, params)
    out = torch.empty(1 + len(w["spec"]["params"]), dtype=torch.float64, device="cuda")
    for _ in range(20):
        G.nll(ev, params, out=out)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(200):
        G.nll(ev, params, out=out)
    b.record()
    torch.cuda.synchronize()
    r = {"events": n, "stream_us": a.elapsed_time(b) * 1e3 / 200, "launch": G.get_launch()}
    if rates:
        r["roofline"] = roofline_8d("c3", "fp32", n, 12, r["stream_us"] * 1e-3, rates, hbm_gbs)
    return r


def formula_vs_builtin(rf, torch):
    """The C3 model (1e7 x 3 FP32 columns) with its Gaussian and Exponential
    written as formula leaves, against the same model with the built-in
    leaves: per-call time of each (the formula graph adds its normalisation
    kernel)."""
    import numpy as np

    w = make_workload("c3")
    spec = w["spec"]
    alt = {**spec, "nodes": [dict(n) for n in spec["nodes"]]}
    for n in alt["nodes"]:
        if n["type"] == "gauss":
            n.update(type="formula", formula="exp(-0.5*((x-p0)/p1)^2)")
        elif n["type"] == "exp":
            n.update(type="formula", formula="exp(p0*x)")
    ev = torch.from_numpy(np.ascontiguousarray(w["cols"])).cuda()
    params = torch.tensor(spec["params"], dtype=torch.float64, device="cuda")
    out = {}
    for tag, sp in (("builtin", spec), ("formula", alt)):
        G = rf.Graph(sp, w["dtype"], "fp32")
        G.tune(ev, params)
        o = torch.empty(1 + len(sp["params"]), dtype=torch.float64, device="cuda")
        for _ in range(10):
            G.nll(ev, params, out=o)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(100):
            G.nll(ev, params, out=o)
        b.record()
        torch.cuda.synchronize()
        out[tag] = {"us_per_call": a.elapsed_time(b) * 10.0, "launches": G.last_launches(),
                    "nll": float(o[0].item())}
    return out


def toy_bench(args, rf, torch, rank, world, pk):
    """--workload c4: a step is one batched NLL + gradient of all 4096 toys."""
    import numpy as np

    import datagen
    w = datagen.c4()
    ev = torch.from_numpy(w["cols"]).cuda()
    off = torch.from_numpy(w["offsets"]).cuda()
    pm = torch.from_numpy(w["params_matrix"]).cuda()
    toys = len(w["offsets"]) - 1
    n = int(w["offsets"][-1])
    G = rf.Graph(w["spec"], "f64", args.precision)
    G.bind_events(ev, toys)
    out = G.nll_batched(off, pm)
    for _ in range(args.warmup):
        G.nll_batched(off, pm, out=out)
    torch.cuda.synchronize()
    uuid = None
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        uuid = u if u.startswith("GPU-") else f"GPU-{u}"
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    time.sleep(0.3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        G.nll_batched(off, pm, out=out)
    b.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(a.elapsed_time(b), dist, "cuda") / args.steps
    # roofline of the step (prep + segment + finalize kernels): the op-list
    # roofline (FP32 evaluation reads the FP32 copy of the columns made once at
    # bind: 4 bytes per event), with the FP32 issue fraction and HBM beside it
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_mhz = float(pk.get("sm_max_mhz") or 2070.0)
    col_bytes = 4 if args.precision == "fp32" else 8
    hbm_gbs = n * col_bytes / (ms * 1e-3) / 1e9
    hbm = {"achieved": hbm_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": hbm_gbs / pk["hbm_gbs"], "peak_source": pk["source"],
           "bytes_per_launch": n * col_bytes}
    traffic = profiled_traffic(G.toy_kernel_hash()) if G.uses_jit() else None
    rates = rf.microbench()
    roofline = {**roofline_8d("c4", args.precision, n, col_bytes, ms, rates, pk["hbm_gbs"]),
                "traffic": traffic, "kernel": "rf_toys_jit (+ prep, finalize)",
                "peak_source": "derived: per-event operation counts x operation rates measured "
                               "alone on this GPU (rf_microbench), HBM bandwidth of "
                               + pk["source"],
                "launch_ms": ms, "hbm": hbm}
    if args.precision == "fp32":
        instr = algorithmic_instr_per_event(w["spec"], REF_EPT, False)
        peak = sms * 128 * sm_mhz * 1e6
        achieved = instr * n / (ms * 1e-3)
        roofline["issue"] = {"achieved": achieved / 1e9, "peak": peak / 1e9,
                             "unit": "G FP32-lane instr/s", "frac": achieved / peak,
                             "instr_per_event": instr,
                             "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x "
                                            f"{sm_mhz:.0f} MHz"}
    line = {"metric": METRIC, "value": job_throughput(n, world, ms), "unit": "events/s",
            "toy_nll_per_s": world * toys / (ms * 1e-3), "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": w["name"], "toys": toys, "events": n,
                       "launch": G.get_toy_launch(), "kernel": G.uses_jit(),
                       "kernel_hash": G.toy_kernel_hash(),
                       "l2": f"inputs larger than L2 ({n * col_bytes / 1e6:.0f} MB > 2 x 129 MB), "
                             "no flush"},
            "clocks": clk,
            "gpu_launches": G.last_launches() * args.steps, "roofline": roofline}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    w = make_workload(args.workload)
    n = w["cols"].shape[1]
    sample = min(n, args.cpu_sample) if args.cpu_sample > 0 else n
    rates = []
    cores = 0
    for _ in range(args.warmup):
        cpu_oracle_rate(w, min(sample, 100_000))
    for _ in range(args.steps):
        r, cores, _ = cpu_oracle_rate(w, sample)
        rates.append(r)
    value = statistics.median(rates)
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "events/s",
            "n_gpus": args.gpus, "gpus_used": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sample / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "events": n, "sample_events": sample},
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"first {sample} of {n} events per step, FP64 NLL + "
                                       "analytic gradient, OpenMP over fixed chunks"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ept", type=int, default=0,
                    help="events per thread of the fused kernel (0: default / tuned)")
    ap.add_argument("--generic", action="store_true",
                    help="run the precompiled generic kernels instead of the per-graph ones")
    ap.add_argument("--min-blocks", type=int, default=0,
                    help="register budget of the specialised kernel (2, 3 or 4; with --no-tune)")
    ap.add_argument("--block", type=int, default=0,
                    help="threads per block of the fused kernel (64, 128 or 256; with --no-tune)")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="grid of the fused kernel in blocks per SM (1..8; with --no-tune)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="events for the CPU oracle baseline (0: the whole workload)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch

    import paper_2003_12875_gb300 as rf

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pk = peaks()

    if args.workload == "c4":
        return toy_bench(args, rf, torch, rank, world, pk)

    # ---------------------------------------------------------------- data
    w = make_workload(args.workload)
    spec = w["spec"]
    n = w["cols"].shape[1]
    col_bytes = 4 if w["dtype"] == "f32" else 8
    host = torch.from_numpy(np.ascontiguousarray(w["cols"]))
    ev = host.cuda()
    params = torch.tensor(spec["params"], dtype=torch.float64, device="cuda")
    G = rf.Graph(spec, w["dtype"], args.precision)
    if args.generic:
        G.set_jit(False)
    out = torch.empty(1 + len(spec["params"]), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    tuned_ms = None
    if args.block:
        G.set_launch(block=args.block)
    if args.ept:
        G.set_launch(ept=args.ept)
    if args.min_blocks:
        G.set_launch(min_blocks=args.min_blocks)
    if args.blocks_per_sm:
        G.set_launch(blocks_per_sm=args.blocks_per_sm)
    if not args.no_tune:
        tuned_ms = G.tune(ev, params)
    for _ in range(args.warmup):
        G.nll(ev, params, out=out)
    torch.cuda.synchronize()

    uuid = None
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        uuid = u if u.startswith("GPU-") else f"GPU-{u}"
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    time.sleep(0.3)

    # ---------------------------------------------------------- timed region
    # Inputs larger than twice the L2 run back to back between two events (a
    # call's FP64 prologue overlaps the previous call's event pass, as in any
    # queue of evaluations); smaller ones get an L2 flush and per-step events.
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    # inputs smaller than twice the L2 are flushed before every step (a
    # 258 MB write, then a 258 MB read of another buffer, outside the per-step
    # events) and the step time is the sum of the per-step events
    in_bytes = n * w["cols"].shape[0] * col_bytes
    flush = L2Flush(torch) if in_bytes < 2 * L2_BYTES else None
    if flush is not None:
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_all0.record(stream)
    if flush is None:
        for i in range(args.steps):
            G.nll(ev, params, out=out)
    else:
        for i in range(args.steps):
            flush()
            starts[i].record(stream)
            G.nll(ev, params, out=out)
            ends[i].record(stream)
    t_all1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    if flush is None:
        total_ms = t_all0.elapsed_time(t_all1)
        launch_ms = [total_ms / args.steps]
    else:
        launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        total_ms = sum(launch_ms)
    per_launch = statistics.mean(launch_ms)
    launches_per_step = G.last_launches()
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_throughput(n, world, ms_per_step)
    nll_value = float(out[0].item())

    # -------------------------------------------------------------- e2e
    pinned = host.pin_memory()
    hp = torch.tensor(spec["params"], dtype=torch.float64)
    G.nll_host(pinned, hp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_nll, _ = G.nll_host(pinned, hp)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e = {"value": world * n / e2e_s, "unit": "events/s",
           "h2d_bytes_per_step": int(host.numel() * col_bytes + 8 * len(spec["params"])),
           "d2h_bytes_per_step": int(8 * (1 + len(spec["params"]))),
           "ms_per_step": e2e_s * 1e3,
           "path": "rf_nll_host on pinned host memory ("
                   + ("staged copy" if os.environ.get("RF_HOST_DIRECT") == "0"
                      else "read in place by the kernel over the host link") + ")"}

    # ----------------------------------------------------------- roofline
    # The roofline of the step (t_roof above: the slower of the event bytes at
    # the measured HBM bandwidth and the per-event operations at their
    # measured rates); per_launch is the time per call (back to back, a call's
    # FP64 prologue overlaps the previous call's event pass).  Beside it: the
    # FP32 issue fraction by this kernel's own instruction count, and HBM.
    bytes_per_launch = n * w["cols"].shape[0] * col_bytes
    hbm_achieved = bytes_per_launch / (per_launch * 1e-3) / 1e9
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = float(pk.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0)
    traffic = profiled_traffic(G.kernel_hash()) if G.uses_jit() else None
    hbm = {"achieved": hbm_achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": hbm_achieved / pk["hbm_gbs"], "peak_source": pk["source"],
           "bytes_per_launch": bytes_per_launch}
    rates = rf.microbench()
    r8 = roofline_8d(args.workload, args.precision, n, w["cols"].shape[0] * col_bytes,
                     per_launch, rates, pk["hbm_gbs"])
    roofline = {**r8, "traffic": traffic, "kernel": "rf_fused_jit (+ prologue)",
                "peak_source": "derived: per-event operation counts x operation rates measured "
                               "alone on this GPU (rf_microbench), HBM bandwidth of "
                               + pk["source"],
                "launch_ms": per_launch, "hbm": hbm}
    if args.precision == "fp32":
        instr = algorithmic_instr_per_event(spec, REF_EPT, w["dtype"] == "f64")
        peak = sms * 128 * sm_mhz * 1e6
        achieved = instr * n / (per_launch * 1e-3)
        roofline["issue"] = {"achieved": achieved / 1e9, "peak": peak / 1e9,
                             "unit": "G FP32-lane instr/s", "frac": achieved / peak,
                             "instr_per_event": instr,
                             "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x "
                                            f"{sm_mhz:.0f} MHz"}

    line = {"metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": w["name"], "events": n, "columns": w["cols"].shape[0],
                       "column_dtype": w["dtype"], "eval": args.precision,
                       "free_params": sum(1 for f in (spec.get("fixed") or []) if not f)
                       or len(spec["params"]),
                       "l2": (f"inputs larger than L2 ({bytes_per_launch / 1e6:.0f} MB > 2 x 129 MB), "
                              "no flush") if flush is None else
                             (f"inputs {bytes_per_launch / 1e6:.1f} MB: L2 flushed before every step "
                              "(258 MB write, then a 258 MB read of another buffer, so "
                              "the write-backs land outside the timed call), step time "
                              "= sum of per-step events"),
                       "launch": G.get_launch(), "tuned_ms": tuned_ms,
                       "kernel": "specialised (NVRTC)" if G.uses_jit() else "generic",
                       "regs_per_thread": G.kernel_regs(),
                       "kernel_hash": G.kernel_hash(),
                       "parallelism": f"{world} independent replica(s)"},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "clocks": clk, "e2e": e2e, "nll": nll_value}

    # ------------------------------------------------------------ extras
    if rank == 0 and world == 1 and not args.no_extras:
        ex = {}
        # fused FP64-eval on the same workload
        G64 = rf.Graph(spec, w["dtype"], "fp64")
        o64 = torch.empty_like(out)
        G64.nll(ev, params, out=o64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            G64.nll(ev, params, out=o64)
        b.record()
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) / 3
        ex["fused_fp64_eval"] = {"events_per_s": n / (t64 * 1e-3), "ms": t64,
                                 "nll": float(o64[0].item()),
                                 "roofline": roofline_8d(args.workload, "fp64", n,
                                                         w["cols"].shape[0] * col_bytes, t64,
                                                         rates, pk["hbm_gbs"])}
        # plain FP64 node-by-node baseline, gradient by central differences
        v, g = G.nll_plain(ev, params)
        torch.cuda.synchronize()
        a.record()
        v, g = G.nll_plain(ev, params)
        b.record()
        torch.cuda.synchronize()
        tp = a.elapsed_time(b)
        ex["plain_fp64"] = {"events_per_s": n / (tp * 1e-3), "ms": tp,
                            "launches": G.last_launches(), "nll": float(v.item()),
                            "fused_speedup": tp / ms_per_step}
        a.record()
        v, _ = G.nll_plain(ev, params, grad=False)
        b.record()
        torch.cuda.synchronize()
        ex["plain_fp64_nll_only_ms"] = a.elapsed_time(b)
        ex["microbench_ops_per_s"] = rates
        ex["small_configs"] = small_configs(rf, torch, rates, pk["hbm_gbs"])
        ex["toys"] = toy_study(rf, torch, rates=rates, hbm_gbs=pk["hbm_gbs"])
        line["extras"] = ex

    if rank == 0 and world == 1 and not args.no_cpu:
        sample = min(n, args.cpu_sample) if args.cpu_sample > 0 else n
        r, cores, dt = cpu_oracle_rate(w, sample)
        line["cpu_baseline"] = {"value": r, "unit": "events/s", "cores": cores, "kind": "oracle",
                                "sample": f"first {sample} of {n} events, one pass, "
                                          f"FP64 NLL + analytic gradient ({dt:.2f} s wall, "
                                          f"{cores} threads)"}
        s1 = min(n, 10_000_000)
        r1, _, dt1 = cpu_oracle_rate(w, s1, nthreads=1)
        line["cpu_baseline"]["single_thread"] = {
            "value": r1, "unit": "events/s", "cores": 1,
            "sample": f"first {s1} of {n} events, one pass ({dt1:.2f} s wall)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
