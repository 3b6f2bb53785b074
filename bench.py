#!/usr/bin/env python3
"""Benchmark: distance-preconditioned Wilson-clover point-source solves on GB300.

Workload (the interacting heavy-quark case): 48x24^3 lattice, antiperiodic
time, synthetic SU(3) links U = exp(i eps H) with eps = 0.3 (seed 1), c_sw =
1.7, M = 0.5, cosh profile alpha_B = 1/cosh[alpha0 (y0 - T/2)] with alpha0 =
0.4, residue r = 1e-11.  One step = one point-source solve: the 12
spin-colour right-hand sides batched in the multi-RHS FP32 inner BiCGStab
inside the FP64 defect-correction loop, then odd-site reconstruction, 1/alpha
restore and the C_PP contraction.  Each step uses a new seeded random source
site.  Metric: solves/s (higher is better).

Also reported: the dslash roofline (HBM) of the dominant kernel, its
A^-1 D launch with all 12 RHS active timed with CUDA events on the
launching stream right after the timed region (the same launches inside the
solve beside it, from CUDA events around every dslash launch of a pass
without graphs), with the DRAM traffic of a stored ncu capture of that
launch shape, labelled as such; the plain single-RHS FP64 GPU solver on the
same workload; the end-to-end number through the host-buffer C-ABI call;
the CPU oracle baseline (a timed full oracle solve of one of the 12
right-hand sides); the cost of the library's per-slice accuracy check
against the paper's global stopping rule alone; the double-float outer
residual; the four-field serving stream (p50/p99 against FP64 plain); and
the SM clocks seen during the timed region.

--gpus N without a torchrun environment starts N local ranks itself (one
per GPU, torch.distributed.run on 127.0.0.1); each rank runs an independent
replica of the workload (no data-path collective).

--impl reference times the CPU oracle (the plain FP64 reference of the
method) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "heavy-quark point-source solve 48x24^3",
    "lattice": [48, 24, 24, 24],
    "bc_t": -1,
    "links": "exp(i eps H), eps=0.3, seed 1 (synthetic; CLS ensembles not available)",
    "csw": 1.7,
    "M": 0.5,
    "profile": "cosh_t alpha0=0.4 (alpha_B = 1/cosh[alpha0 (y0 - T/2)])",
    "residue": 1e-11,
    "rhs_per_solve": 12,
}
# per-run state of the benchmark (clock samples, the tune cache); git-ignored
STATE = os.environ.get("DP_BENCH_STATE", os.path.join(ROOT, ".bench_state"))
DIMS = (48, 24, 24, 24)
EPS, SEED, CSW, MASS, ALPHA0, RES = 0.3, 1, 1.7, 0.5, 0.4, 1e-11
METRIC = "Precond. Wilson-clover solves/s & dslash HBM GB/s vs FP64 plain; p99 latency"
UNIT = "solves/s"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_tune_cache(path):
    """Launch shapes from an earlier run ({"TxLxLxL prec_nN": [block, rpt, stages]})."""
    if not path or path == "none" or not os.path.exists(path):
        return {}
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_tune_cache(path, cache):
    if not path or path == "none":
        return
    try:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(cache, fh, indent=1)
    except OSError:
        pass


def rank_max(pg, x):
    """The maximum of a float over the ranks of the job (x itself without a
    process group); NCCL reduces on the GPU, gloo on the host."""
    if pg is None:
        return float(x)
    import torch

    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(steps, ws, ms_max):
    """Whole-job throughput of N independent replicas: the solves of every
    rank over the slowest rank's time (weak scaling)."""
    return steps * ws / (ms_max / 1e3)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(STATE, "bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_solve_sample():
    """Time the CPU oracle on a bounded sample of the workload: one full
    BiCGStab solve of one of the 12 right-hand sides (source component 0 at
    the origin) to the benchmark's residue.  Returns (seconds, iterations,
    threads)."""
    import lattice_inputs as li
    import oracle

    U = li.su3_links(DIMS, EPS, SEED)
    op = oracle.WilsonClover(U, DIMS, CSW, -1)
    del U
    prof = ("cosh_t", ALPHA0, (0, 0, 0, 0))
    al = oracle.profile_alpha("cosh_t", ALPHA0, DIMS)
    eta = oracle.point_sources(DIMS, (0, 0, 0, 0), al[0][0])[:1]
    op.apply(eta, MASS, prof)  # builds the clover matrices outside the timing
    t0 = time.perf_counter()
    _, iters, _, _ = op.solve(eta, MASS, prof, tol=RES)
    return time.perf_counter() - t0, int(iters[0]), oracle.num_threads()


def oracle_iters_per_rhs():
    """Oracle BiCGStab iterations per RHS on this workload at the benchmark's
    residue, from a stored oracle run under tests/golden (written by the
    oracle only); else the stored count at the tighter residue 1e-13."""
    p = os.path.join(ROOT, "tests", "golden", "oracle_iters_48x24_r1e-11.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["iters"]), "stored oracle run of one RHS at r = %g" % d["tol"]
    p = os.path.join(ROOT, "tests", "golden", "cpp_48x24_M0.5_cosh0.4.json")
    if os.path.exists(p):
        d = json.load(open(p))
        it = d.get("oracle_iters")
        if it:
            return float(np.mean(it)), ("stored oracle run at r = %g (tighter than the "
                                        "benchmark's 1e-11: overstates the CPU time)"
                                        % d.get("tol", 0))
    return None, None


C5_FIELDS = [((16, 8, 8, 8), 0.3, 101), ((32, 16, 16, 16), 0.4, 102),
             ((48, 24, 24, 24), 0.45, 103), ((64, 32, 32, 32), 0.5, 104)]


def c5_profile(M):
    """The serving mix's profile per request: heavy (M >= 0.3) cosh-t with
    alpha0 = 0.4, light cosh-4d with alpha0 = 0.2 (the library's per-slice
    check keeps either accurate to T/2)."""
    return ("cosh_t", 0.4) if M >= 0.3 else ("cosh_4d", 0.2)


def serve_c5(dp, ctx, n_req, loads, n_burst=24, n_fp64=24, seed=2024):
    """Serving stream against 4 resident synthetic gauge fields of mixed
    volumes (16x8^3, 32x16^3, 48x24^3, 64x32^3; eps 0.3, 0.4, 0.45, 0.5;
    seeds 101-104; c_sw 1.7).  Each request draws a field and a source site
    uniformly, M ~ U[0.01, 0.8], the heavy or light profile of c5_profile and
    r = 1e-10 with the library's default per-slice accuracy target.  A closed
    burst of n_burst requests measures the scheduler's capacity; then n_req
    requests arrive as a Poisson stream at each load x that capacity (p50/p99
    latency from submit to completion).  The plain single-RHS FP64 GPU solver
    serves n_fp64 requests of the same mix one after another (its solves/s).
    Served results of a sample (two per field) are compared per time slice
    with the same request solved to r = 1e-13 through the batched FP64 path
    with another profile (an exact transform of the same system)."""
    import lattice_inputs as li

    fields = []
    for dims, eps, sd in C5_FIELDS:
        U = li.su3_links(dims, eps, sd)
        f = dp.dp_field_load(ctx, U, dims, -1)
        del U
        dp.dp_field_set_csw(ctx, f, 1.7)
        dp.dp_autotune(ctx, f, "mixed_fp32", 1, 48)
        fields.append((f, dims))
    rng = np.random.default_rng(seed)

    def draw(k=None):
        k = int(rng.integers(0, 4)) if k is None else k
        f, dims = fields[k]
        M = float(rng.uniform(0.01, 0.8))
        src = tuple(int(rng.integers(0, d)) for d in dims)
        return k, f, dims, M, c5_profile(M), src

    budget = int(200e9)  # of the 288 GB; fields and four 48-slot batches take ~140 GB
    dp.dp_trim(ctx)
    dp.dp_serve_start(ctx, budget, 48)
    t0 = time.perf_counter()
    # the burst and the plain FP64 sample take the four fields equally often
    # (each request's cost depends on its volume by two decades)
    order = [k % 4 for k in range(n_burst)]
    rng.shuffle(order)
    tk = [(dp.dp_submit(ctx, r[1], r[3], r[4], r[5], 1e-10), r) for r in (draw(k) for k in order)]
    for t, r in tk:
        dp.dp_wait(ctx, t, r[2][0], timeout_s=1200)
    cap = n_burst / (time.perf_counter() - t0)
    dp.dp_serve_stop(ctx, True)
    legs = []
    for load in loads:
        rate = cap * load
        dp.dp_serve_start(ctx, budget, 48)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
        reqs = []
        t0 = time.perf_counter()
        for k in range(n_req):
            while time.perf_counter() - t0 < arrivals[k]:
                time.sleep(min(0.002, max(0.0, arrivals[k] - (time.perf_counter() - t0))))
            r = draw()
            reqs.append((dp.dp_submit(ctx, r[1], r[3], r[4], r[5], 1e-10), r))
        bad, refined, worst = 0, 0, 0.0
        for t, r in reqs:
            _, info = dp.dp_wait(ctx, t, r[2][0], timeout_s=1200)
            bad += info["status"] != 0
            refined += info["refine_rounds"] > 0
            worst = max(worst, info["slice_residue"])
        st = dp.dp_serve_stats_get(ctx)
        dp.dp_serve_stop(ctx, True)
        legs.append({"offered_load": load, "offered_rate_per_s": rate, "requests": n_req,
                     "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                     "solves_per_s": st["solves_per_s"], "not_ok": bad,
                     "refined_requests": refined, "slice_residue_max": worst,
                     "max_concurrent_batches": st["max_concurrent_batches"],
                     "wall_s": time.perf_counter() - t0})
    # the plain single-RHS FP64 solver on the same mix, one request at a time
    o64 = {"prec": "fp64", "batched": 0, "use_graph": 0, "max_iter": 400000}
    t64, n64_bad = 0.0, 0
    for i in range(n_fp64):
        _, f, dims, M, prof, src = draw(i % 4)
        (_, _, i64), dt = _timed(lambda: dp.dp_solve_point(ctx, f, M, prof, src, 1e-10, o64, T=dims[0]))
        t64 += dt
        n64_bad += i64["status"] != 0
    fp64_rate = n_fp64 / t64
    # accuracy of served results: two requests per field
    errs, sample = [], []
    dp.dp_serve_start(ctx, budget, 48)
    o_ref = {"prec": "fp64", "batched": 1, "use_graph": 0}
    for k in [0, 1, 2, 3, 0, 1, 2, 3]:
        _, f, dims, M, prof, src = draw(k)
        t = dp.dp_submit(ctx, f, M, prof, src, 1e-10)
        cpp_served, info = dp.dp_wait(ctx, t, dims[0], timeout_s=1200)
        ref_prof = ("cosh_t", 0.6)
        tight = dp.dp_solve_point(ctx, f, M, ref_prof, src, 1e-13, o_ref, T=dims[0])[0]
        e = slice_err(cpp_served, tight, dims[0] // 2)
        errs.append(e)
        sample.append({"dims": list(dims), "M": M, "profile": list(prof), "served_vs_tight_to_T2": e,
                       "refine_rounds": info["refine_rounds"], "slice_residue": info["slice_residue"]})
    dp.dp_serve_stop(ctx, True)
    for f, _ in fields:
        dp.dp_field_free(ctx, f)
    dp.dp_trim(ctx)
    return {"workload": "serving stream, 4 resident fields (16x8^3, 32x16^3, 48x24^3, 64x32^3)",
            "capacity_requests_per_s": cap, "burst_requests": n_burst, "legs": legs,
            "fp64_plain": {"solves_per_s": fp64_rate, "requests": n_fp64, "not_ok": n64_bad},
            "capacity_over_fp64_plain": cap / fp64_rate,
            "served_per_slice_rel_err_vs_tight_max_to_T2": max(errs), "accuracy_sample": sample,
            "mix": "field and source uniform; M ~ U[0.01, 0.8]; heavy (M >= 0.3) cosh-t alpha0 = 0.4, "
                   "light cosh-4d alpha0 = 0.2; r = 1e-10 with the default per-slice target; up to "
                   "4 requests (48 RHS) per field batch, one stream and worker per field"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    iters, src = oracle_iters_per_rhs()
    if iters is None:
        iters, src = 100.0, "assumed 100 iterations per RHS (no stored oracle run)"
    # warm-up (also builds the clover matrices)
    import lattice_inputs as li

    U = li.su3_links(DIMS, EPS, SEED)
    op = oracle.WilsonClover(U, DIMS, CSW, -1)
    psi = li.random_spinor(DIMS, 1, 5)
    prof = ("cosh_t", ALPHA0, (0, 0, 0, 0))
    for _ in range(args.warmup):
        op.apply(psi, MASS, prof)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        op.apply(psi, MASS, prof)
    dt = (time.perf_counter() - t0) / args.steps
    per_solve = dt * 2 * iters * 12
    value = 1.0 / per_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "extrapolated, not a timed solve: one full-lattice (D'+M) "
                                   "application on 1 RHS per step; a solve = 12 RHS x 2 "
                                   "applications x %.0f BiCGStab iterations (%s)"
                                   % (iters, src)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


LINKS = {"mixed_fp32": "12-real FP32 links", "mixed_fp16": "12-real FP16 links + FP32 scale",
         "mixed_bf16": "12-real BF16 links + FP32 scale"}


# ---- the other workloads of the study (each prints one JSON line) ----------
def heavy_or_light(M):
    """Profile per mass: heavy (M >= 0.3) cosh-t with alpha0 = min(ln(1+M), 0.5)
    rounded as 0.4 / 0.5; light cosh-4d with alpha0 = 0.2."""
    if M >= 0.3:
        return ("cosh_t", 0.4 if M < 0.65 else 0.5)
    return ("cosh_4d", 0.2)


def slice_err(cpp, ref, upto):
    c, r = np.asarray(cpp)[: upto + 1], np.asarray(ref)[: upto + 1]
    return float(np.max(np.abs(c / r - 1)))


def oracle_dslash_rate(U, dims, csw, M, prof, reps=3):
    """The CPU oracle's full-lattice (D+M) application on one RHS at this
    volume, timed on the host cores (a reported baseline): ms per
    application, sites/s, and GB/s of algorithmic bytes V x (48 + 72 + 72)
    x 8 (spinor in and out, the 4 links of a site read once as 18 reals
    each, 72 reals of clover per site)."""
    import lattice_inputs as li
    import oracle

    op = oracle.WilsonClover(U, dims, csw, -1)
    psi = li.random_spinor(dims, 1, 5)
    p3 = (prof[0], prof[1], (0, 0, 0, 0))
    op.apply(psi, M, p3)  # builds the clover matrices outside the timing
    t0 = time.perf_counter()
    for _ in range(reps):
        op.apply(psi, M, p3)
    dt = (time.perf_counter() - t0) / reps
    V = int(np.prod(dims))
    return op, {"ms_per_application": dt * 1e3, "sites_per_s": V / dt,
                "algorithmic_gbs": V * (48 + 72 + 72) * 8 / dt / 1e9,
                "cores": oracle.num_threads(), "kind": "oracle"}


def _timed(fn):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def config_free16(dp, ctx, args):
    """Free theory 16x8^3 (U = 1), antiperiodic time, M = 0.5, exp profile
    alpha0 = 0.4, origin source, r = 1e-11; C_PP against the exact
    momentum-space values stored under tests/golden."""
    import lattice_inputs as li

    dims = (16, 8, 8, 8)
    f = dp.dp_field_load(ctx, li.unit_links(dims), dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "free_16x8_M0.5.json")))["cpp"]
    res = {}
    for name, o in (("fp64_plain", {"prec": "fp64", "batched": 0, "use_graph": 0}),
                    ("mixed_batched", {"prec": "mixed_fp32", "batched": 1, "use_graph": 1})):
        for _ in range(args.warmup):
            dp.dp_solve_point(ctx, f, 0.5, ("exp_t", 0.4), (0, 0, 0, 0), 1e-11, o, T=16)
        ts = []
        for _ in range(args.steps):
            (cpp, _, info), dt = _timed(
                lambda: dp.dp_solve_point(ctx, f, 0.5, ("exp_t", 0.4), (0, 0, 0, 0), 1e-11, o, T=16))
            ts.append(dt)
        meff = [float(np.log(cpp[t] / cpp[t + 1])) for t in range(8)]
        res[name] = {"solves_per_s": 1.0 / float(np.median(ts)), "ms_per_solve": 1e3 * float(np.median(ts)),
                     "iters_inner": info["iters_inner"], "iters_outer": info["iters_outer"],
                     "true_rel_residue": info["true_rel_residue"],
                     "per_slice_rel_err_vs_exact_max_to_T2": slice_err(cpp, gold, 8),
                     "per_slice_rel_err_vs_exact_all": slice_err(cpp, gold, 15),
                     "effective_mass_0_7": meff}
    dp.dp_field_free(ctx, f)
    # the CPU oracle on the whole workload (12 components, FP64 BiCGStab)
    import oracle

    op, rate = oracle_dslash_rate(li.unit_links(dims), dims, 1.7, 0.5, ("exp_t", 0.4))
    t0 = time.perf_counter()
    cpp_o, _, oinfo = oracle.solve_point(op, 0.5, "exp_t", 0.4, (0, 0, 0, 0), tol=1e-11)
    to = time.perf_counter() - t0
    res["cpu_baseline"] = {"value": 1.0 / to, "unit": "solves/s", "cores": oracle.num_threads(),
                           "kind": "oracle", "sample": "the whole workload: one solve of all 12 "
                           "components to r = 1e-11, %.2f s" % to,
                           "per_slice_rel_err_vs_exact_max_to_T2": slice_err(cpp_o, gold, 8),
                           "dslash": rate}
    return {"workload": "free theory 16x8^3 (U = 1), M = 0.5, exp_t alpha0 = 0.4, r = 1e-11",
            "reference": "exact momentum-space C_PP (tests/golden/free_16x8_M0.5.json)", **res}


def config_light64(dp, ctx, args):
    """Light quarks on 64x32^3 (eps = 0.5, seed 7, c_sw = 1.9): M in {0.02,
    0.01, 0.005}, cosh-4d profile alpha0 in {0 (unpreconditioned), 0.2, 0.4},
    16-bit (FP16) links in the FP32 inner solver, FP64 outer loop, r = 1e-10.
    Iteration counts and solves/s under the paper's global stopping rule (the
    per-slice residual reported, not refined), the restored C_PP of the
    preconditioned solves against the unpreconditioned one; then the same
    M = 0.005 solves with the library's default per-slice target against the
    stored oracle result (tests/golden, written by the oracle only)."""
    import lattice_inputs as li

    dims = (64, 32, 32, 32)
    U = li.su3_links(dims, 0.5, 7)
    f = dp.dp_field_load(ctx, U, dims, -1)
    # the CPU oracle's operator at this volume (a full solve of one RHS of
    # the light quark takes minutes on the host; the application rate is the
    # reported baseline)
    _, oracle_rate = oracle_dslash_rate(U, dims, 1.9, 0.005, ("cosh_4d", 0.2), reps=2)
    del U
    dp.dp_field_set_csw(ctx, f, 1.9)
    prec = args.prec if args.prec != "mixed_fp32" else "mixed_fp16"
    dp.dp_autotune(ctx, f, prec, 1, 12)
    dp.dp_autotune(ctx, f, "fp64", 0, 12)
    o = {"prec": prec, "batched": 1, "use_graph": 1, "max_iter": 40000}
    o_paper = dict(o, slice_tol=1e30)  # the per-slice residual measured, never refined
    rows = []
    src = (0, 0, 0, 0)
    dp.dp_solve_point(ctx, f, 0.02, ("cosh_4d", 0.2), src, 1e-10, o_paper, T=64)  # warm-up
    for M in (0.02, 0.01, 0.005):
        base = None
        for a0 in (0.0, 0.2, 0.4):
            prof = ("none", 0.0) if a0 == 0 else ("cosh_4d", a0)
            (cpp, _, info), dt = _timed(lambda: dp.dp_solve_point(ctx, f, M, prof, src, 1e-10, o_paper,
                                                                  T=64))
            row = {"M": M, "alpha0": a0, "profile": prof[0], "iters_inner": info["iters_inner"],
                   "iters_outer": info["iters_outer"], "true_rel_residue": info["true_rel_residue"],
                   "slice_residue": info["slice_residue"], "status": info["status"], "seconds": dt}
            if base is None:
                base = cpp
            else:
                dev = np.abs(np.asarray(cpp)[:33] / np.asarray(base)[:33] - 1)
                row["cpp_rel_diff_vs_unprec_max_to_T2"] = float(dev.max())
                over = np.nonzero(dev > 1e-6)[0]
                row["first_slice_over_1e-6"] = int(over[0]) if len(over) else None
            rows.append(row)
    # the library's per-slice target (default) at M = 0.005 against the oracle
    checked = []
    gold = os.path.join(ROOT, "tests", "golden", "cpp_64x32_M0.005.json")
    ref = np.asarray(json.load(open(gold))["masses"][0]["cpp"]) if os.path.exists(gold) else None
    for a0, pr in ((0.0, prec), (0.2, prec), (0.4, prec), (0.2, "mixed_fp32")):
        prof = ("none", 0.0) if a0 == 0 else ("cosh_4d", a0)
        oo = dict(o, prec=pr)
        (cpp, _, info), dt = _timed(lambda: dp.dp_solve_point(ctx, f, 0.005, prof, src, 1e-10, oo, T=64))
        row = {"M": 0.005, "alpha0": a0, "profile": prof[0], "inner": pr,
               "iters_inner": info["iters_inner"], "iters_outer": info["iters_outer"],
               "refine_rounds": info["refine_rounds"], "slice_residue": info["slice_residue"],
               "status": info["status"], "seconds": dt}
        if ref is not None:
            row["per_slice_rel_err_vs_oracle_max_to_T2"] = slice_err(cpp, ref, 32)
        checked.append(row)
    # the paper's Table I comparison with its own solver: SAP+GCR iterations
    # against alpha0 (FP32 links, r = 1e-10)
    sap_rows = []
    for ncy in (4, 2):
        for a0 in (0.0, 0.2, 0.4):
            prof = ("none", 0.0) if a0 == 0 else ("cosh_4d", a0)
            osap = {"prec": "mixed_fp32", "solver": "sap_gcr", "batched": 1, "use_graph": 0,
                    "sap_ncy": ncy, "sap_nmr": 4, "gcr_nkv": 8, "max_iter": 4000,
                    "slice_tol": 1e30}
            (cpp, _, info), dt = _timed(lambda: dp.dp_solve_point(ctx, f, 0.005, prof, src, 1e-10, osap,
                                                                  T=64))
            sap_rows.append({"M": 0.005, "alpha0": a0, "sap_ncy": ncy, "gcr_iters": info["iters_inner"],
                             "iters_outer": info["iters_outer"], "status": info["status"],
                             "true_rel_residue": info["true_rel_residue"], "seconds": dt})
    dp.dp_field_free(ctx, f)
    return {"workload": "light-quark solves 64x32^3 (eps 0.5, seed 7, c_sw 1.9), r = 1e-10",
            "sap_gcr": sap_rows,
            "inner": "%s (%s) in FP64 defect correction" % (prec, LINKS[prec]), "solves": rows,
            "per_slice_checked": checked, "cpu_oracle_dslash": oracle_rate}


def config_multimass32(dp, ctx, args):
    """32x16^3 (eps = 0.4, seed 3, c_sw = 1.7), one point source, 12 RHS x 4
    masses {0.01, 0.1, 0.5, 0.8} each with its own profile, one 48-RHS batch:
    default vs autotuned launch shapes, CUDA graphs on and off, and the
    12-RHS FP32 dslash against the HBM roofline."""
    import torch

    import lattice_inputs as li

    import oracle

    dims = (32, 16, 16, 16)
    U = li.su3_links(dims, 0.4, 3)
    f = dp.dp_field_load(ctx, U, dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    Ms = [0.01, 0.1, 0.5, 0.8]
    profs = [heavy_or_light(M) for M in Ms]
    # the CPU oracle on a bounded sample: its operator at this volume, and
    # one full solve of one RHS (component 0, the heavy mass 0.5) to the
    # workload's residue, scaled to one mass x 12 RHS
    op, rate = oracle_dslash_rate(U, dims, 1.7, 0.5, heavy_or_light(0.5))
    del U
    hp = heavy_or_light(0.5)
    al = oracle.profile_alpha(hp[0], hp[1], dims, (3, 5, 7, 9))
    eta = oracle.point_sources(dims, (3, 5, 7, 9), al[0][3] * al[1][5] * al[2][7] * al[3][9])[:1]
    t0 = time.perf_counter()
    _, oit, _, _ = op.solve(eta, 0.5, (hp[0], hp[1], (3, 5, 7, 9)), tol=1e-10)
    to = time.perf_counter() - t0
    del op
    cpu = {"value": 1.0 / (12 * to), "unit": "solves/s (one mass x 12 RHS)",
           "cores": oracle.num_threads(), "kind": "oracle",
           "sample": "one full oracle BiCGStab solve of 1 of the 12 RHS of M = 0.5 to r = 1e-10 "
                     "(%.1f s, %d iterations), x 12" % (to, int(oit[0])), "dslash": rate}
    out = torch.zeros(4 * 32, dtype=torch.float64, device="cuda")
    src = (3, 5, 7, 9)
    res = {}

    def run(label, graphs):
        o = {"prec": "mixed_fp32", "compress12": 1, "batched": 1, "use_graph": graphs}
        for _ in range(max(1, args.warmup)):
            dp.dp_solve_point_dev(ctx, f, Ms, profs, src, 1e-10, out.data_ptr(), o)
        ts = []
        for _ in range(args.steps):
            infos, dt = _timed(lambda: dp.dp_solve_point_dev(ctx, f, Ms, profs, src, 1e-10,
                                                             out.data_ptr(), o))
            ts.append(dt)
        res[label] = {"ms_per_48rhs_solve": 1e3 * float(np.median(ts)),
                      "solves_per_s": 4.0 / float(np.median(ts)),
                      "iters_inner": [i["iters_inner"] for i in infos],
                      "true_rel_residue_max": max(i["true_rel_residue"] for i in infos)}

    run("fixed_shape_graphs", 1)
    shape = dp.dp_autotune(ctx, f, "mixed_fp32", 1, 48)
    dp.dp_autotune(ctx, f, "fp64", 0, 48)
    run("autotuned_graphs", 1)
    run("autotuned_no_graphs", 0)
    res["tuned_shape_48rhs"] = {"block": shape[0], "rhs_per_thread": shape[1], "stages": shape[2],
                                "ms": shape[3]}
    # 12-RHS FP32 dslash in isolation: default vs tuned shape
    nb = dp.dp_spinor_bytes(ctx, f, "mixed_fp32", 12)
    a = torch.randn(nb // 4, device="cuda")
    b = torch.empty_like(a)
    Vh = int(np.prod(dims)) // 2
    byt = Vh * (12 * 48 * 4 + 8 * 48 + 72 * 4)
    hbm, src_pk = peaks()
    for label, kw in (("dslash12_fixed", dict(block_threads=64, rhs_per_thread=2, stages=0)),
                      ("dslash12_tuned", dict(block_threads=0, rhs_per_thread=0, stages=-1))):
        if label == "dslash12_tuned":
            dp.dp_autotune(ctx, f, "mixed_fp32", 1, 12)
        dp.dp_dslash_dev(ctx, f, 0.5, ("cosh_t", 0.4), "mixed_fp32", 1, 0, a.data_ptr(), b.data_ptr(),
                         12, iters=5, **kw)
        ms = dp.dp_dslash_dev(ctx, f, 0.5, ("cosh_t", 0.4), "mixed_fp32", 1, 0, a.data_ptr(),
                              b.data_ptr(), 12, iters=50, **kw)
        res[label] = {"avg_launch_ms": ms, "achieved_gbs": byt / (ms / 1e3) / 1e9,
                      "frac_of_hbm": byt / (ms / 1e3) / 1e9 / hbm, "peak_source": src_pk,
                      "note": "inputs %d MB > 129 MB L2 only in part at this volume" % (nb >> 20)}
    dp.dp_field_free(ctx, f)
    return {"workload": "multi-mass 32x16^3 (eps 0.4, seed 3), 12 RHS x 4 masses in one batch, "
                        "r = 1e-10", "masses": Ms, "profiles": [list(p) for p in profs],
            "cpu_baseline": cpu, **res}


def config_sf48(dp, ctx, args):
    """Dirichlet time boundary (the Schroedinger-functional-like setting of
    the end of Sec. II) on 48x24^3 (eps = 0.3, seed 1, c_sw = 1.7), heavy
    quark M = 0.5, source on the first time slice: the correlator falls over
    the whole time extent.  Unpreconditioned and exp-profile (alpha0 = 0.4)
    solves at the loose residue r = 1e-6 against a tight (r = 1e-12)
    reference, per time slice over all 48 slices, under the paper's global
    stopping rule (per-slice residual reported, not refined) and with the
    library's default per-slice target."""
    import lattice_inputs as li

    dims = (48, 24, 24, 24)
    f = dp.dp_field_load(ctx, li.su3_links(dims, 0.3, 1), dims, 0)
    dp.dp_field_set_csw(ctx, f, 1.7)
    dp.dp_autotune(ctx, f, "mixed_fp32", 1, 12)
    o = {"prec": "mixed_fp32", "batched": 1, "use_graph": 1}
    src = (0, 0, 0, 0)
    ref, _, iref = dp.dp_solve_point(ctx, f, 0.5, ("exp_t", 0.4), src, 1e-12,
                                     dict(o, slice_tol=1e-11), T=48)
    rows = []
    # (global only: the per-slice check off; far slices the loose solve has
    # not reached would otherwise still be refined)
    for check in ("global only", "default per-slice target"):
        oc = dict(o, slice_tol=-1.0) if check == "global only" else o
        for prof, r in ((("none", 0.0), 1e-6), (("exp_t", 0.4), 1e-6), (("none", 0.0), 1e-11),
                        (("exp_t", 0.4), 1e-11)):
            (cpp, _, info), dt = _timed(lambda: dp.dp_solve_point(ctx, f, 0.5, prof, src, r, oc, T=48))
            dev = np.abs(np.asarray(cpp) / np.asarray(ref) - 1)
            over = np.nonzero(dev > 1e-6)[0]
            rows.append({"check": check, "profile": list(prof), "r": r,
                         "iters_inner": info["iters_inner"], "iters_outer": info["iters_outer"],
                         "refine_rounds": info["refine_rounds"],
                         "slice_residue": info["slice_residue"], "status": info["status"],
                         "seconds": dt, "per_slice_rel_dev_max_all_slices": float(dev.max()),
                         "first_slice_over_1e-6": int(over[0]) if len(over) else None})
    dp.dp_field_free(ctx, f)
    return {"workload": "Dirichlet-time heavy quark 48x24^3 (eps 0.3, seed 1), M = 0.5, source on "
                        "slice 0", "reference": "exp_t alpha0 = 0.4 at r = 1e-12",
            "cpp_ref_0_over_47": float(ref[0] / ref[47]), "solves": rows}


def config_heavy48grid(dp, ctx, args):
    """The heavy-quark grid on 48x24^3 (eps = 0.3, seed 1, c_sw = 1.7, origin
    source): M in {0.5, 0.8} x cosh-t alpha0 in {0 (unpreconditioned), 0.3,
    0.4, 0.5} x r in {1e-6, 1e-11}, all 12 RHS batched, in FP64 and in the
    FP32-inner / FP64-outer mixed precision, under the paper's global
    stopping rule alone (Sec. I); per time slice to T/2, C_PP against the
    unpreconditioned FP64 solve of the same mass at r = 1e-12 held to a
    per-slice target of 1e-11.  The mixed solves at r = 1e-6 are repeated
    with the library's default per-slice target."""
    import lattice_inputs as li

    dims = (48, 24, 24, 24)
    T = dims[0]
    f = dp.dp_field_load(ctx, li.su3_links(dims, 0.3, 1), dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    dp.dp_autotune(ctx, f, "mixed_fp32", 1, 12)
    src = (0, 0, 0, 0)
    precs = {"fp64": {"prec": "fp64", "batched": 1, "use_graph": 0},
             "mixed_fp32": {"prec": "mixed_fp32", "compress12": 1, "batched": 1, "use_graph": 1}}
    rows, refs = [], {}
    for M in (0.5, 0.8):
        ref, _, iref = dp.dp_solve_point(ctx, f, M, ("none", 0.0), src, 1e-12,
                                         dict(precs["fp64"], slice_tol=1e-11), T=T)
        refs[str(M)] = {"status": iref["status"], "slice_residue": iref["slice_residue"],
                        "cpp_0_over_T2": float(ref[0] / ref[T // 2])}
        cases = [(p, a0, r, -1.0) for p in precs for a0 in (0.0, 0.3, 0.4, 0.5)
                 for r in (1e-6, 1e-11)]
        cases += [("mixed_fp32", a0, 1e-6, 0.0) for a0 in (0.0, 0.3, 0.4, 0.5)]
        for prec, a0, r, stol in cases:
            prof = ("none", 0.0) if a0 == 0 else ("cosh_t", a0)
            o = dict(precs[prec], slice_tol=stol)
            (cpp, _, info), dt = _timed(lambda: dp.dp_solve_point(ctx, f, M, prof, src, r, o, T=T))
            dev = np.abs(np.asarray(cpp)[: T // 2 + 1] / np.asarray(ref)[: T // 2 + 1] - 1)
            over = np.nonzero(dev > 1e-6)[0]
            rows.append({"M": M, "prec": prec, "alpha0": a0, "r": r,
                         "check": "global only" if stol < 0 else "default per-slice target",
                         "iters_inner": info["iters_inner"], "iters_outer": info["iters_outer"],
                         "refine_rounds": info["refine_rounds"],
                         "slice_residue": info["slice_residue"], "status": info["status"],
                         "seconds": dt, "per_slice_rel_dev_max_to_T2": float(dev.max()),
                         "first_slice_over_1e-6": int(over[0]) if len(over) else None})
    dp.dp_field_free(ctx, f)
    return {"workload": "heavy quark 48x24^3 (eps 0.3, seed 1, c_sw 1.7), origin source, "
                        "12 RHS batched", "reference": "unpreconditioned FP64 at r = 1e-12, "
                        "per-slice target 1e-11", "references": refs, "solves": rows}


def config_serve(dp, ctx, args):
    """The four-field serving stream (serve_c5) at 0.5x, 0.9x and 1.2x the
    measured capacity."""
    return serve_c5(dp, ctx, args.serve_requests, (0.5, 0.9, 1.2))


def run_config(args):
    import torch

    import paper_1006_4028_gb300 as dp

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    dp.load()
    ctx = dp.dp_create(0, torch.cuda.current_stream().cuda_stream)
    fn = {"free16": config_free16, "light64": config_light64, "multimass32": config_multimass32,
          "serve": config_serve, "sf48": config_sf48,
          "heavy48grid": config_heavy48grid}[args.config]
    t0 = time.perf_counter()
    line = fn(dp, ctx, args)
    line = {"config_mode": args.config, "wall_s": time.perf_counter() - t0, **line}
    dp.dp_destroy(ctx)
    print(json.dumps(line), flush=True)
    return 0


def spawn_local_ranks(n):
    """Start n local ranks of this same command (one per GPU) when bench.py
    was not launched by torchrun; each rank runs an independent replica."""
    import socket

    import torch

    if torch.cuda.device_count() < n:
        print("bench.py --gpus %d: only %d CUDA devices visible" % (n, torch.cuda.device_count()),
              file=sys.stderr)
        return 2
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node",
           str(n), "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-plain", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-df", action="store_true",
                    help="skip the leg with the outer Schur operator in double-float")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="requests of the Poisson serving stream (per offered load)")
    ap.add_argument("--serve-load", type=float, default=0.9,
                    help="offered load of the serving leg as a fraction of the capacity a closed burst of the same request mix measures")
    ap.add_argument("--dims", default=None,
                    help="T,Lx,Ly,Lz of a smaller lattice for profiling runs (not the headline)")
    ap.add_argument("--prec", default="mixed_fp32",
                    choices=["mixed_fp32", "mixed_fp16", "mixed_bf16"],
                    help="inner-solver precision (links: 12 FP32 reals, or 12 16-bit reals "
                         "plus one FP32 scale)")
    ap.add_argument("--solver", default="bicgstab", choices=["bicgstab", "cgne", "sap_gcr"])
    ap.add_argument("--config", default="heavy48",
                    choices=["heavy48", "heavy48grid", "free16", "light64", "multimass32", "serve",
                             "sf48"],
                    help="heavy48: the headline solves/s line (default); the others run the "
                         "study's other workloads and print their own JSON line")
    ap.add_argument("--tune-cache", default=os.path.join(STATE, "tunecache.json"),
                    help="launch shapes kept between runs of a workload ('none': always tune)")
    ap.add_argument("--graphs", type=int, default=1,
                    help="capture solver iterations as CUDA graphs in the timed region (the "
                         "per-kernel event times then come from a separate pass of up to 3 "
                         "solves without graphs)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return spawn_local_ranks(args.gpus)
    if args.dims:
        global DIMS
        DIMS = tuple(int(v) for v in args.dims.split(","))
        WORKLOAD["lattice"] = list(DIMS)
        WORKLOAD["workload"] = "heavy-quark point-source solve %dx%d^3 (profiling size)" % (
            DIMS[0], DIMS[1])
        args.no_cpu_baseline = True
    if args.impl == "reference":
        return run_reference(args)
    if args.config != "heavy48":
        return run_config(args)

    ws, rank, local = dist_env()
    import torch

    import lattice_inputs as li
    import paper_1006_4028_gb300 as dp

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
        pg = tdist
    dp.load()
    stream = torch.cuda.current_stream()
    ctx = dp.dp_create(local, stream.cuda_stream)
    U = li.su3_links(DIMS, EPS, SEED)
    field = dp.dp_field_load(ctx, U, DIMS, -1)
    dp.dp_field_set_csw(ctx, field, CSW)
    del U
    T, V = DIMS[0], int(np.prod(DIMS))
    opts = {"prec": args.prec, "compress12": 1, "batched": 1, "use_graph": args.graphs,
            "solver": args.solver}
    link_bytes = 48 if args.prec == "mixed_fp32" else 28  # per link in the inner dslash
    prof = ("cosh_t", ALPHA0)
    rng = np.random.default_rng(1000 + rank)

    def rand_src():
        return tuple(int(rng.integers(0, d)) for d in DIMS)

    # tune the launch shapes of the dslash for this volume and batch, or take
    # them from the tune cache an earlier run of this workload wrote (so that
    # a rerun under a profiler launches the same kernels)
    tuned = {}
    cache = load_tune_cache(args.tune_cache)
    for prec, c12, nrs in ((args.prec, 1, (12,)), ("fp64", 0, (12, 1))):
        for nr in nrs:
            key = "%s_n%d" % (prec, nr)
            ckey = "%s %s" % ("x".join(map(str, DIMS)), key)
            if ckey in cache:
                try:
                    dp.dp_tune_set(ctx, field, prec, c12, nr, *cache[ckey][:3])
                    tuned[key] = list(cache[ckey][:3]) + ["from tune cache"]
                    continue
                except dp.DpError:
                    pass
            tuned[key] = dp.dp_autotune(ctx, field, prec, c12, nr)
            cache[ckey] = list(tuned[key][:3])
    if rank == 0:
        save_tune_cache(args.tune_cache, cache)

    cpp_dev = torch.zeros(T, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES, cpp_dev.data_ptr(), opts)
    torch.cuda.synchronize()

    # ---- timed region: K solves, inputs resident in HBM ----
    # per-kernel CUDA events are recorded around every launch of the timed
    # region, unless the solver iterations run as CUDA graphs (events cannot
    # be read per launch inside a replayed graph): then a separate pass with
    # events and without graphs measures the kernels
    dp.dp_timing_reset(ctx)
    dp.dp_timing_enable(ctx, not args.graphs)
    clk = Clocks(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clk.start()
    n0 = dp.dp_launch_count(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos += dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES,
                                       cpp_dev.data_ptr(), opts)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop()
    launches = dp.dp_launch_count(ctx) - n0
    ms = e0.elapsed_time(e1)
    kernel_timing_region = "timed region"
    if args.graphs:
        kernel_timing_region = "instrumented pass of %d solves without graphs" % min(args.steps, 3)
        dp.dp_timing_enable(ctx, True)
        o_ng = dict(opts, use_graph=0)
        ms_ng0 = torch.cuda.Event(enable_timing=True)
        ms_ng1 = torch.cuda.Event(enable_timing=True)
        ms_ng0.record(stream)
        for _ in range(min(args.steps, 3)):
            dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES, cpp_dev.data_ptr(),
                                  o_ng)
        ms_ng1.record(stream)
        torch.cuda.synchronize()
        ms_instr = ms_ng0.elapsed_time(ms_ng1)
    else:
        ms_instr = ms
    d32_n, d32_ms = dp.dp_timing_get(ctx, "dslash_fp32")
    d64_n, d64_ms = dp.dp_timing_get(ctx, "dslash_fp64")
    dp.dp_timing_enable(ctx, False)
    ms = rank_max(pg, ms)
    value = replica_value(args.steps, ws, ms)

    # ---- roofline of the dominant kernel (multi-RHS FP32 dslash) ----
    Vh = V // 2
    n = 12
    # algorithmic bytes per half-site: spinor in/out n*(24+24)*4, 8 links
    # (12 FP32 reals, or 12 16-bit reals + an FP32 scale), the FP32 clover
    # inverse (72 reals); the second Schur launch also reads x (n*24*4):
    # average of the two launch kinds
    b_ainv = n * 48 * 4 + 8 * link_bytes + 72 * 4
    b_xmy = b_ainv + n * 24 * 4
    bytes_per_launch = Vh * (b_ainv + b_xmy) / 2
    avg_ms = d32_ms / max(d32_n, 1)
    hbm_peak, peak_src = peaks()
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    # cross-check: the same kernel with all 12 RHS active, timed in isolation
    buf_in = torch.zeros(dp.dp_spinor_bytes(ctx, field, args.prec, 12) // 4, dtype=torch.float32,
                         device="cuda")
    buf_in.normal_()
    buf_out = torch.empty_like(buf_in)
    iso_ms = dp.dp_dslash_dev(ctx, field, MASS, prof, args.prec, 1, 0, buf_in.data_ptr(),
                              buf_out.data_ptr(), 12, 0, 0, 20)
    del buf_in, buf_out
    iso_gbs = Vh * b_ainv / (iso_ms / 1e3) / 1e9
    # the same kernel against the FP32 ALUs: n*(1320 + 96) flop per half-site
    # for the hops with their profile factors, ~504 per RHS for the fused
    # A^-1, ~24 per RHS for x - ... in the second Schur launch; peak = SMs x
    # 128 FP32 lanes x 2 flop x the maximum SM clock (a packed f32x2 FMA
    # issues two of those lanes' work, it does not add lanes)
    # (the A^-1 D launch timed with all RHS active, as the headline roofline)
    flop_ainv = n * (1320 + 96 + 504)
    flop_per_launch = Vh * flop_ainv
    props = torch.cuda.get_device_properties(local)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    alu = {"bound": "alu", "achieved": flop_per_launch / (iso_ms / 1e3) / 1e12,
           "peak": fp32_peak, "unit": "TFLOP/s",
           "frac": flop_per_launch / (iso_ms / 1e3) / 1e12 / fp32_peak,
           "flop_per_launch": flop_per_launch,
           "peak_source": "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (maximum SM clock)"
                          % (props.multi_processor_count, sm_max)}

    # DRAM bytes of one launch of the tuned kernel, from an ncu capture of this
    # workload (dram__bytes_read.sum + dram__bytes_write.sum, median of 12
    # autotuner launches of the A^-1 D kernel with all 12 RHS active, 12-real
    # FP32 links), per launch shape (threads per block, RHS per thread,
    # stages); valid only while the tuner picks a captured shape
    captured = {(64, 2, 2): 1000676992, (96, 2, 2): 999261184, (64, 2, 5): 999319936,
                (64, 2, 6): 1029303296, (128, 2, 6): 1027006976}
    traffic, traffic_note = None, "tuned shape has no ncu capture"
    shape = tuple(tuned.get("%s_n12" % args.prec, [0, 0, 0])[:3])
    if args.prec == "mixed_fp32" and shape in captured and DIMS == (48, 24, 24, 24):
        traffic = captured[shape]
        traffic_note = ("stored, not measured in this run: ncu dram__bytes_read.sum + "
                        "dram__bytes_write.sum of one A^-1 D launch of shape %s at 48x24^3 "
                        "(median of 12 autotuner launches, all 12 RHS active; algorithmic "
                        "%.0f bytes), captured with the kernel as it is now"
                        % (list(shape), Vh * b_ainv))
    # ---- end to end: host-buffer C-ABI call per solve (wall clock) ----
    e2e_steps = max(3, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cpp_h = None
    for _ in range(e2e_steps):
        cpp_h, _, info_h = dp.dp_solve_point(ctx, field, MASS, prof, rand_src(), RES, opts, T=T)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    # every rank serves its own requests: the job's rate is the solves of all
    # ranks over the slowest rank's time, as for the device-timed value
    e2e_s = rank_max(pg, e2e_s)
    Lm = max(DIMS)
    h2d = 4 * Lm * 8 + 8 * Lm * 8 + 8 * Lm * 4 + 4 + 12 * 40 + 12 * 88 + 12 * 4
    d2h = T * 8

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer",
        "data": "synthetic",
        "config": dict(WORKLOAD, parallelism="replicas" if ws > 1 else "single",
                       l2="working set ~%.1f GB >> 129 MB L2 (no flush needed)"
                          % (dp.dp_device_bytes(ctx) / 1e9),
                       solver="%s FP32 inner (%s) in FP64 defect correction"
                              % ({"bicgstab": "BiCGStab", "cgne": "CGNE", "sap_gcr": "SAP+GCR"}[args.solver],
                                 LINKS[args.prec]),
                       graphs=bool(args.graphs), tuned_launch=tuned),
        "gpu_launches": launches,
        "iterations": {"inner_mean": float(np.mean([i["iters_inner"] for i in infos])),
                       "outer_mean": float(np.mean([i["iters_outer"] for i in infos])),
                       "true_rel_residue_max": float(max(i["true_rel_residue"] for i in infos)),
                       "slice_residue_max": float(max(i["slice_residue"] for i in infos)),
                       "refine_rounds_mean": float(np.mean([i["refine_rounds"] for i in infos]))},
        "roofline": {"bound": "hbm", "achieved": iso_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": iso_gbs / hbm_peak, "traffic": traffic,
                     "traffic_note": traffic_note,
                     "kernel": "dslash_fp32 A^-1 D (12 RHS, %s, fused A^-1 epilogue), the solver's "
                               "launch shape" % LINKS[args.prec],
                     "bytes_per_launch": Vh * b_ainv, "avg_launch_ms": iso_ms, "launches": 20,
                     "peak_source": peak_src,
                     "measured_in": "20 launches with all 12 RHS active, CUDA events on the "
                                    "launching stream, in this benchmark process after the timed "
                                    "region",
                     "in_solve": {"achieved": achieved, "frac": achieved / hbm_peak,
                                  "avg_launch_ms": avg_ms, "launches": d32_n,
                                  "bytes_per_launch": bytes_per_launch,
                                  "measured_in": kernel_timing_region,
                                  "note": "bytes count all 12 RHS in every launch; converged RHS "
                                          "are masked out of the last launches of each inner "
                                          "solve, so this overstates the bytes moved"},
                     "fp32_alu": alu},
        "kernel_time_share": {"dslash_fp32": d32_ms / ms_instr, "dslash_fp64": d64_ms / ms_instr},
        "clocks": clocks,
        "e2e": {"value": ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": "dp_solve_point with host buffers; request parameters and profile "
                        "tables up, C_PP down"},
    }

    if rank == 0 and not args.no_fp64_plain:
        o64 = {"prec": "fp64", "batched": 0, "use_graph": 0}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, i64 = dp.dp_solve_point(ctx, field, MASS, prof, rand_src(), RES, o64, T=T)
        s64 = time.perf_counter() - t0
        line["fp64_plain"] = {"solves_per_s": 1.0 / s64, "ms_per_solve": s64 * 1e3,
                              "iters_inner": i64["iters_inner"],
                              "speedup_of_value": value / ws * s64}
    if rank == 0:
        # the paper's global stopping rule alone (the library's per-slice
        # accuracy check off): what the check costs on this workload
        # (slice_tol = 1e30: the check runs and reports the worst slice but
        # never refines)
        o_g = dict(opts, slice_tol=1e30)
        dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES, cpp_dev.data_ptr(), o_g)
        torch.cuda.synchronize()
        k_g = max(3, min(args.steps, 5))
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        ig = []
        for _ in range(k_g):
            ig += dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES,
                                        cpp_dev.data_ptr(), o_g)
        g1.record(stream)
        torch.cuda.synchronize()
        line["global_criterion_only"] = {
            "solves_per_s": 1e3 * k_g / g0.elapsed_time(g1),
            "iters_inner": float(np.mean([i["iters_inner"] for i in ig])),
            "outer": float(np.mean([i["iters_outer"] for i in ig])),
            "slice_residue_max": float(max(i["slice_residue"] for i in ig)),
            "note": "the paper's global residue test alone: the per-slice residual measured "
                    "(slice_tol 1e30), no refinement"}
    if rank == 0 and not args.no_df:
        # the same solves with the outer loop's Schur operator in double-float
        # (two FP32 per real) instead of FP64
        o_df = dict(opts, outer_df=1)
        for _ in range(2):
            dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES, cpp_dev.data_ptr(), o_df)
        torch.cuda.synchronize()
        k_df = max(3, min(args.steps, 5))
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        idf = []
        for _ in range(k_df):
            idf += dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES, cpp_dev.data_ptr(),
                                         o_df)
        d1.record(stream)
        torch.cuda.synchronize()
        ms_df = d0.elapsed_time(d1) / k_df
        # kernel times of the outer operator, FP64 vs double-float (one
        # instrumented solve each)
        dp.dp_timing_reset(ctx)
        dp.dp_timing_enable(ctx, True)
        dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES, cpp_dev.data_ptr(),
                              dict(o_df, use_graph=0))
        dp.dp_solve_point_dev(ctx, field, [MASS], [prof], rand_src(), RES, cpp_dev.data_ptr(),
                              dict(opts, use_graph=0))
        torch.cuda.synchronize()
        ndf, tdf = dp.dp_timing_get(ctx, "dslash_df")
        n64, t64_ = dp.dp_timing_get(ctx, "dslash_fp64")
        dp.dp_timing_enable(ctx, False)
        line["outer_double_float"] = {
            "outer_operator_ms": {"double_float_two_launches": tdf / max(ndf, 1),
                                  "fp64_two_launches": t64_ / max(n64, 1) * 2},
            "solves_per_s": 1e3 / ms_df, "ms_per_solve": ms_df,
            "iters_inner": float(np.mean([i["iters_inner"] for i in idf])),
            "outer": float(np.mean([i["iters_outer"] for i in idf])),
            "true_rel_residue_max": float(max(i["true_rel_residue"] for i in idf))}
    if rank == 0 and not args.no_cpu_baseline:
        secs, iters, thr = cpu_solve_sample()
        line["cpu_baseline"] = {
            "value": 1.0 / (12 * secs), "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": "one full oracle BiCGStab solve (timed, %.1f s, %d iterations) of 1 of "
                      "the 12 right-hand sides (component 0, source at the origin) to r = %g; "
                      "a solve = 12 such right-hand sides" % (secs, iters, RES)}
    # parity of one solve at the origin source against the stored oracle result
    gold = os.path.join(ROOT, "tests", "golden", "cpp_48x24_M0.5_cosh0.4.json")
    if rank == 0 and os.path.exists(gold) and DIMS == (48, 24, 24, 24):
        g = json.load(open(gold))
        c, _, _ = dp.dp_solve_point(ctx, field, MASS, prof, (0, 0, 0, 0), RES, opts, T=T)
        ref = np.asarray(g["cpp"])
        line["per_slice_rel_err_vs_oracle_max"] = float(np.max(np.abs(c[:T // 2 + 1] /
                                                                      ref[:T // 2 + 1] - 1)))
        if "global_criterion_only" in line:
            c, _, _ = dp.dp_solve_point(ctx, field, MASS, prof, (0, 0, 0, 0), RES,
                                        dict(opts, slice_tol=1e30), T=T)
            line["global_criterion_only"]["per_slice_rel_err_vs_oracle_max"] = float(
                np.max(np.abs(c[:T // 2 + 1] / ref[:T // 2 + 1] - 1)))
        # C_AP from the same propagator and the PCAC mass (host ratio)
        cpp_c, cap_c, _ = dp.dp_solve_point_corr(ctx, field, MASS, prof, (0, 0, 0, 0), RES, opts, T=T)
        mp = dp.dp_pcac_mass(cpp_c, cap_c)
        line["pcac_mass_plateau_y0_8_20"] = float(np.mean(mp[8:21]))
        # effective mass of the same C_PP: cosh form and a two-sided fit
        meff = dp.dp_effective_mass(cpp_c, "cosh")
        m_fit, _, rms_fit = dp.dp_fit_correlator(cpp_c, "cosh", 12, 24)
        line["effective_mass"] = {"cosh_y0_8_20": [float(v) for v in meff[8:21]],
                                  "cosh_fit_y0_12_24": m_fit, "fit_rms_rel_dev": rms_fit}
        if "outer_double_float" in line:
            c, _, _ = dp.dp_solve_point(ctx, field, MASS, prof, (0, 0, 0, 0), RES,
                                        dict(opts, outer_df=1), T=T)
            line["outer_double_float"]["per_slice_rel_err_vs_oracle_max"] = float(
                np.max(np.abs(c[:T // 2 + 1] / ref[:T // 2 + 1] - 1)))
    # serving: Poisson arrivals on the resident field through the
    # continuous-batching scheduler; latency from submit to completion
    if rank == 0 and not args.no_serve:
        dp.dp_field_free(ctx, field)
        field = None
        line["serving"] = serve_c5(dp, ctx, args.serve_requests, (args.serve_load,))
    if field is not None:
        dp.dp_field_free(ctx, field)
    dp.dp_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
