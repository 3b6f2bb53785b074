"""Write stored oracle results used by the GPU tests and the benchmark.

Calls only the CPU oracle (and the seeded input generators).  Each output is
a JSON file in this directory with the inputs that produced it.

  cpp_48x24_M0.5_cosh0.4.json : C_PP(y0) of the point source at the origin on
      the 48x24^3 heavy-quark workload (eps = 0.3, seed 1, c_sw = 1.7,
      antiperiodic time, M = 0.5, cosh profile alpha0 = 0.4), solved by the
      oracle's full-lattice FP64 BiCGStab to relative residue 1e-13, restored
      (Sec. II eq. backcorrection), plus the oracle's iteration counts.

  free_16x8_M0.5.json : C_PP(y0) of the free theory (U = 1) on 16x8^3,
      antiperiodic time, M = 0.5, from the exact momentum-space propagator
      (no solve; it is independent of any profile after the restore).

  cpp_64x32_M0.005.json : C_PP(y0) of the point source at the origin on the
      64x32^3 light-quark workload (eps = 0.5, seed 7, c_sw = 1.9,
      antiperiodic time, M = 0.005), solved by the oracle's full-lattice FP64
      BiCGStab to 1e-13 with the time profile cosh_t alpha0 = 0.4 (the result
      does not depend on the profile after the restore; this one keeps the
      far slices of S' within a few decades of the near ones, so the global
      residue bounds them too), plus the oracle's per-slice residuals of the
      restored solution on the unpreconditioned system.

  cpp_32x16_multimass.json : the same for the 32x16^3 multi-mass workload
      (eps = 0.4, seed 3, c_sw = 1.7, M in {0.01, 0.1, 0.5, 0.8}).

  oracle_iters_48x24_r1e-11.json : the oracle's BiCGStab iteration count for
      one right-hand side of the 48x24^3 heavy-quark workload at r = 1e-11.

Run:  python tests/golden/make_golden.py [heavy|free|light64|multimass32|iters48]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import lattice_inputs as li  # noqa: E402
import oracle  # noqa: E402


def heavy_48x24():
    dims = (48, 24, 24, 24)
    eps, seed, csw, M, alpha0, tol = 0.3, 1, 1.7, 0.5, 0.4, 1e-13
    t0 = time.time()
    U = li.su3_links(dims, eps, seed)
    op = oracle.WilsonClover(U, dims, csw, -1)
    cpp, _, info = oracle.solve_point(op, M, "cosh_t", alpha0, (0, 0, 0, 0), tol=tol)
    out = {
        "what": "oracle C_PP(y0), point source at the origin, restored",
        "dims": list(dims), "eps": eps, "seed": seed, "csw": csw, "bc_t": -1, "M": M,
        "profile": "cosh_t", "alpha0": alpha0, "src": [0, 0, 0, 0], "tol": tol,
        "cpp": [float(v) for v in cpp],
        "oracle_iters": [int(v) for v in info["iters"]],
        "oracle_relres": [float(v) for v in info["relres"]],
        "converged": bool(info["converged"]),
        "oracle_threads": oracle.num_threads(),
        "seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, "cpp_48x24_M0.5_cosh0.4.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def _certified(dims, eps, seed, csw, masses, name, alpha0=0.4, tol=1e-13):
    t0 = time.time()
    U = li.su3_links(dims, eps, seed)
    op = oracle.WilsonClover(U, dims, csw, -1)
    del U
    out = {
        "what": "oracle C_PP(y0), point source at the origin, restored; slice_residual = "
                "max over y0 of |eta - (D+M) S|_t / |S|_t on the unpreconditioned system",
        "dims": list(dims), "eps": eps, "seed": seed, "csw": csw, "bc_t": -1,
        "profile": "cosh_t", "alpha0": alpha0, "src": [0, 0, 0, 0], "tol": tol,
        "masses": [], "oracle_threads": oracle.num_threads(),
    }
    for M in masses:
        cpp, S, info = oracle.solve_point(op, M, "cosh_t", alpha0, (0, 0, 0, 0), tol=tol)
        eta = oracle.point_sources(dims, (0, 0, 0, 0))
        rho = oracle.slice_residuals(op, M, S, eta, 0)
        del S, eta, info["Sprime"]
        out["masses"].append({
            "M": M, "cpp": [float(v) for v in cpp],
            "slice_residual": [float(v) for v in rho],
            "oracle_iters": [int(v) for v in info["iters"]],
            "oracle_relres": [float(v) for v in info["relres"]],
            "converged": bool(info["converged"]),
        })
        out["seconds"] = time.time() - t0
        with open(os.path.join(HERE, name), "w") as fh:
            json.dump(out, fh, indent=1)


def light_64x32():
    _certified((64, 32, 32, 32), 0.5, 7, 1.9, [0.005], "cpp_64x32_M0.005.json")


def multimass_32x16():
    _certified((32, 16, 16, 16), 0.4, 3, 1.7, [0.01, 0.1, 0.5, 0.8], "cpp_32x16_multimass.json")


def iters_48x24():
    """Oracle BiCGStab iterations of one right-hand side (source component 0
    at the origin) of the 48x24^3 heavy-quark workload to r = 1e-11, the
    benchmark's residue (the reference arm's iteration count)."""
    dims = (48, 24, 24, 24)
    eps, seed, csw, M, alpha0, tol = 0.3, 1, 1.7, 0.5, 0.4, 1e-11
    U = li.su3_links(dims, eps, seed)
    op = oracle.WilsonClover(U, dims, csw, -1)
    al = oracle.profile_alpha("cosh_t", alpha0, dims)
    eta = oracle.point_sources(dims, (0, 0, 0, 0), al[0][0])[:1]
    t0 = time.time()
    _, iters, rel, ok = op.solve(eta, M, ("cosh_t", alpha0, (0, 0, 0, 0)), tol=tol)
    out = {"what": "oracle BiCGStab iterations, one RHS (component 0, origin source)",
           "dims": list(dims), "eps": eps, "seed": seed, "csw": csw, "M": M,
           "profile": "cosh_t", "alpha0": alpha0, "tol": tol, "iters": int(iters[0]),
           "relres": float(rel[0]), "converged": bool(ok), "seconds": time.time() - t0,
           "oracle_threads": oracle.num_threads()}
    with open(os.path.join(HERE, "oracle_iters_48x24_r1e-11.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def free_16x8():
    dims, M = (16, 8, 8, 8), 0.5
    cpp = oracle.free_cpp(dims, M, -1)
    out = {
        "what": "exact momentum-space free C_PP(y0), point source at the origin",
        "dims": list(dims), "bc_t": -1, "M": M, "cpp": [float(v) for v in cpp],
    }
    with open(os.path.join(HERE, "free_16x8_M0.5.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    which = sys.argv[1:] or ["heavy", "free"]
    if "free" in which:
        free_16x8()
    if "heavy" in which:
        heavy_48x24()
    if "multimass32" in which:
        multimass_32x16()
    if "light64" in which:
        light_64x32()
    if "iters48" in which:
        iters_48x24()
