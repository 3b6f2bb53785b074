"""Python binding of libdpre, the GB300 library for distance-preconditioned
Wilson-clover solves (arXiv 1006.4028).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libdpre.so`` (built in-tree by :mod:`.build`).  The functions keep
the names of the C ABI declared in ``include/dpre.h``.  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.

Host arrays use numpy complex128 in the lexicographic layouts of the header:
links ``(T, Lz, Ly, Lx, 4, 3, 3)``, spinors ``(nrhs, T, Lz, Ly, Lx, 4, 3)``.
Profiles are given as ``(kind, alpha0)`` or ``(kind, alpha0, tables)`` with
kind one of ``"none", "exp_t", "cosh_t", "cosh_4d", "table"`` (alpha_B
orientation: S' = alpha_B S, see the header).

A point-source solve, restored and contracted::

    import paper_1006_4028_gb300 as dp
    ctx = dp.dp_create(0)
    f = dp.dp_field_load(ctx, links, (48, 24, 24, 24), -1)   # antiperiodic time
    dp.dp_field_set_csw(ctx, f, 1.7)
    dp.dp_autotune(ctx, f, "mixed_fp32", 1, 12)               # optional
    cpp, _, info = dp.dp_solve_point(ctx, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-11,
                                     {"prec": "mixed_fp32"}, T=48)
    m_eff = dp.dp_effective_mass(cpp, "cosh")
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "DpError", "load", "lib_path",
    "dp_create", "dp_destroy", "dp_last_error", "dp_device_bytes", "dp_trim",
    "dp_field_load", "dp_field_set_csw", "dp_field_free",
    "dp_solve_point", "dp_solve_point_multi", "dp_solve_point_dev",
    "dp_solve_point_corr", "dp_solve_point_hl", "dp_pcac_mass", "dp_effective_mass", "dp_fit_correlator", "dp_apply", "dp_profile_tables", "dp_spinor_bytes", "dp_dslash_dev", "dp_schur_dev",
    "dp_autotune", "dp_tune_set",
    "dp_timing_enable", "dp_timing_reset", "dp_timing_get", "dp_launch_count",
    "dp_serve_start", "dp_submit", "dp_wait", "dp_cancel", "dp_serve_stats_get", "dp_serve_stop",
    "PROFILE_KINDS", "PREC", "SOLVER", "APPLY", "STATUS", "MEFF_KINDS",
]

PROFILE_KINDS = {"none": 0, "exp_t": 1, "cosh_t": 2, "cosh_4d": 3, "table": 4}
PREC = {"fp64": 0, "mixed_fp32": 1, "mixed_fp16": 2, "mixed_bf16": 3}
SOLVER = {"bicgstab": 0, "cgne": 1, "sap_gcr": 2}
APPLY = {"hop": 0, "clover": 1, "full": 2, "clover_inv": 3}
STATUS = {0: "DP_OK", 1: "DP_ERR_INVALID_ARG", 2: "DP_ERR_OOM", 3: "DP_ERR_NOT_CONVERGED",
          4: "DP_ERR_BREAKDOWN", 5: "DP_ERR_NONFINITE", 6: "DP_ERR_TIMEOUT", 7: "DP_ERR_REJECTED",
          8: "DP_ERR_CUDA", 9: "DP_ERR_NOT_FOUND"}


class DpError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status
        self.message = message


class Profile(C.Structure):
    _fields_ = [("kind", C.c_int), ("alpha0", C.c_double), ("table", C.POINTER(C.c_double) * 4)]


class SolveOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("solver", C.c_int), ("prec", C.c_int),
                ("compress12", C.c_int), ("inner_tol", C.c_double), ("batched", C.c_int),
                ("use_graph", C.c_int), ("check_every", C.c_int), ("sap_ncy", C.c_int),
                ("sap_nmr", C.c_int), ("gcr_nkv", C.c_int), ("outer_df", C.c_int),
                ("slice_tol", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters_inner", C.c_int), ("iters_outer", C.c_int),
                ("true_rel_residue", C.c_double), ("seconds", C.c_double),
                ("n_rhs", C.c_int), ("status", C.c_int), ("slice_residue", C.c_double),
                ("refine_rounds", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(C.Structure):
    _fields_ = [("field", C.c_uint64), ("M", C.c_double), ("profile", Profile),
                ("src", C.c_int * 4), ("r", C.c_double), ("prec", C.c_int),
                ("slice_tol", C.c_double)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_long), ("completed", C.c_long), ("rejected", C.c_long),
                ("in_flight", C.c_long), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("mean_ms", C.c_double), ("solves_per_s", C.c_double),
                ("hbm_budget", C.c_size_t), ("hbm_in_use", C.c_size_t),
                ("max_concurrent_batches", C.c_int), ("yields", C.c_long)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libdpre.so (raises if it has not been built and building is off)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise ImportError("libdpre.so is not built (%s); run paper_1006_4028_gb300.build.build()"
                              % _build.LIB)
        _build.build()
    lib = C.CDLL(_build.LIB)
    vp, ip, dp, up, sz = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_size_t
    P = C.POINTER
    sig = {
        "dp_create": ([P(vp), ip, vp, vp], ip),
        "dp_destroy": ([vp], None),
        "dp_last_error": ([], C.c_char_p),
        "dp_device_bytes": ([vp], sz),
        "dp_trim": ([vp], ip),
        "dp_effective_mass": ([vp, ip, ip, vp], ip),
        "dp_pcac_mass": ([vp, vp, ip, vp], ip),
        "dp_fit_correlator": ([vp, ip, ip, ip, ip, P(dp), P(dp), P(dp)], ip),
        "dp_field_load": ([vp, vp, P(C.c_int * 4), ip, P(up)], ip),
        "dp_field_set_csw": ([vp, up, dp], ip),
        "dp_field_free": ([vp, up], ip),
        "dp_solve_point": ([vp, up, dp, P(Profile), P(C.c_int * 4), dp, P(SolveOpts), vp, vp,
                            P(SolveInfo)], ip),
        "dp_solve_point_multi": ([vp, up, ip, vp, vp, P(C.c_int * 4), dp, P(SolveOpts), vp, vp,
                                  vp], ip),
        "dp_solve_point_dev": ([vp, up, ip, vp, vp, P(C.c_int * 4), dp, P(SolveOpts), vp, vp], ip),
        "dp_solve_point_corr": ([vp, up, dp, P(Profile), P(C.c_int * 4), dp, P(SolveOpts), vp, vp,
                                 P(SolveInfo)], ip),
        "dp_solve_point_hl": ([vp, up, dp, P(Profile), dp, P(Profile), P(C.c_int * 4), dp,
                               P(SolveOpts), vp, vp, vp], ip),
        "dp_apply": ([vp, up, ip, dp, P(Profile), P(C.c_int * 4), ip, ip, vp, vp, ip], ip),
        "dp_profile_tables": ([P(C.c_int * 4), ip, P(Profile), P(C.c_int * 4), vp, vp], ip),
        "dp_restore_contract_dev": ([vp, up, ip, vp, vp, vp, vp, vp], ip),
        "dp_restore_contract_noalloc": ([vp, up, ip, vp, vp, vp, vp, vp], ip),
        "dp_spinor_bytes": ([vp, up, ip, ip], sz),
        "dp_schur_dev": ([vp, up, dp, P(Profile), P(C.c_int * 4), ip, ip, ip, ip, vp, vp, ip], ip),
        "dp_dslash_dev": ([vp, up, dp, P(Profile), ip, ip, ip, vp, vp, ip, ip, ip, ip, ip,
                           P(C.c_float)], ip),
        "dp_tune_set": ([vp, up, ip, ip, ip, ip, ip, ip], ip),
        "dp_autotune": ([vp, up, ip, ip, ip, P(C.c_int), P(C.c_int), P(C.c_int), P(C.c_float)],
                        ip),
        "dp_timing_enable": ([vp, ip], ip),
        "dp_timing_reset": ([vp], ip),
        "dp_timing_get": ([vp, C.c_char_p, P(C.c_long), P(C.c_double)], ip),
        "dp_launch_count": ([vp], C.c_long),
        "dp_serve_start": ([vp, sz, ip], ip),
        "dp_submit": ([vp, P(Request), P(up)], ip),
        "dp_wait": ([vp, up, dp, vp, P(SolveInfo)], ip),
        "dp_cancel": ([vp, up], ip),
        "dp_serve_stats_get": ([vp, P(ServeStats)], ip),
        "dp_serve_stop": ([vp, ip], ip),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def dp_last_error():
    return load().dp_last_error().decode(errors="replace")


def _check(st, allow=()):
    if st != 0 and st not in allow:
        raise DpError(st, dp_last_error())
    return st


def _ptr(a):
    return C.c_void_p(a.ctypes.data)


def _profile(p, dims=None):
    """(kind, alpha0[, tables]) -> (Profile, keepalive)."""
    pr = Profile()
    keep = []
    if p is None:
        p = ("none", 0.0)
    kind = p[0]
    pr.kind = PROFILE_KINDS[kind] if isinstance(kind, str) else int(kind)
    pr.alpha0 = float(p[1]) if len(p) > 1 else 0.0
    if len(p) > 2 and p[2] is not None:
        for mu in range(4):
            t = np.ascontiguousarray(p[2][mu], dtype=np.float64)
            keep.append(t)
            pr.table[mu] = t.ctypes.data_as(C.POINTER(C.c_double))
    return pr, keep


def _opts(o):
    s = SolveOpts()
    o = dict(o or {})
    s.max_iter = int(o.get("max_iter", 0))
    sv = o.get("solver", "bicgstab")
    s.solver = SOLVER[sv] if isinstance(sv, str) else int(sv)
    prec = o.get("prec", "mixed_fp32")
    s.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    s.compress12 = int(o.get("compress12", 1))
    s.inner_tol = float(o.get("inner_tol", 0.0))
    s.batched = int(o.get("batched", 1))
    s.use_graph = int(o.get("use_graph", 1))
    s.check_every = int(o.get("check_every", 0))
    s.outer_df = int(o.get("outer_df", 0))
    s.sap_ncy = int(o.get("sap_ncy", 0))
    s.sap_nmr = int(o.get("sap_nmr", 0))
    s.gcr_nkv = int(o.get("gcr_nkv", 0))
    s.slice_tol = float(o.get("slice_tol", 0.0))
    return s


def _i4(v):
    return (C.c_int * 4)(*[int(x) for x in v])


# ---- context --------------------------------------------------------------
def dp_create(device=0, stream=None):
    """Create a context; `stream` is a cudaStream_t handle (int) or None."""
    lib = load()
    h = C.c_void_p()
    _check(lib.dp_create(C.byref(h), int(device), None, C.c_void_p(stream) if stream else None))
    return h


def dp_destroy(ctx):
    load().dp_destroy(ctx)


def dp_device_bytes(ctx):
    return int(load().dp_device_bytes(ctx))


def dp_trim(ctx):
    """Return the device memory the context's pool keeps reserved."""
    _check(load().dp_trim(ctx))


# ---- fields -----------------------------------------------------------------
def dp_field_load(ctx, links, dims, bc_t=-1):
    U = np.ascontiguousarray(links, dtype=np.complex128)
    T, Lx, Ly, Lz = (int(d) for d in dims)
    if U.size != T * Lx * Ly * Lz * 36:
        raise ValueError("links must hold V*4*3*3 complex entries")
    f = C.c_uint64()
    _check(load().dp_field_load(ctx, _ptr(U), C.byref(_i4(dims)), int(bc_t), C.byref(f)))
    return f.value


def dp_field_set_csw(ctx, field, csw):
    _check(load().dp_field_set_csw(ctx, int(field), float(csw)))


def dp_field_free(ctx, field):
    _check(load().dp_field_free(ctx, int(field)))


# ---- solves -------------------------------------------------------------------
def dp_solve_point(ctx, field, M, profile, src, r, opts=None, T=None, V=None, want_prop=False,
                   allow=(3,)):
    """Point-source solve for 12 spin-colour RHS.  Returns (cpp[T], prop, info).

    `T` (and `V` if want_prop) give the lattice sizes of the field.
    """
    pr, keep = _profile(profile)
    cpp = np.zeros(int(T))
    prop = np.zeros((12, int(V), 4, 3), np.complex128) if want_prop else None
    info = SolveInfo()
    o = _opts(opts)
    st = load().dp_solve_point(ctx, int(field), float(M), C.byref(pr), C.byref(_i4(src)), float(r),
                               C.byref(o), _ptr(cpp), _ptr(prop) if want_prop else None,
                               C.byref(info))
    _check(st, allow)
    return cpp, prop, info.as_dict()


def dp_solve_point_corr(ctx, field, M, profile, src, r, opts=None, T=None, allow=(3,)):
    """Point-source solve returning C_PP and C_AP: (cpp[T], cap[T], info)."""
    pr, keep = _profile(profile)
    cpp = np.zeros(int(T))
    cap = np.zeros(int(T))
    info = SolveInfo()
    st = load().dp_solve_point_corr(ctx, int(field), float(M), C.byref(pr), C.byref(_i4(src)),
                                    float(r), C.byref(_opts(opts)), _ptr(cpp), _ptr(cap),
                                    C.byref(info))
    _check(st, allow)
    return cpp, cap, info.as_dict()


def dp_solve_point_hl(ctx, field, Mh, prof_h, Ml, prof_l, src, r, opts=None, T=None,
                      allow=(3,)):
    """Heavy and light quark from one source: (cpp[2, T], hl[T] complex, [info h, info l])."""
    ph, kh = _profile(prof_h)
    pl, kl = _profile(prof_l)
    cpp = np.zeros((2, int(T)))
    hl = np.zeros((int(T), 2))
    infos = (SolveInfo * 2)()
    st = load().dp_solve_point_hl(ctx, int(field), float(Mh), C.byref(ph), float(Ml), C.byref(pl),
                                  C.byref(_i4(src)), float(r), C.byref(_opts(opts)), _ptr(cpp), _ptr(hl),
                                  infos)
    _check(st, allow)
    return cpp, hl[:, 0] + 1j * hl[:, 1], [infos[0].as_dict(), infos[1].as_dict()]


def dp_pcac_mass(cpp, cap):
    """m_PCAC(y0) = [C_AP(y0+1) - C_AP(y0-1)] / (4 C_PP(y0)) for y0 = 1..T-2 (host
    function of the library); NaN at the ends."""
    c = np.ascontiguousarray(cpp, dtype=np.float64)
    a = np.ascontiguousarray(cap, dtype=np.float64)
    if a.shape != c.shape:
        raise ValueError("cpp and cap must have the same length")
    out = np.empty(len(c), dtype=np.float64)
    _check(load().dp_pcac_mass(c.ctypes.data, a.ctypes.data, len(c), out.ctypes.data))
    return out


MEFF_KINDS = {"log": 0, "cosh": 1}


def dp_effective_mass(cpp, kind="log"):
    """Effective mass per y0 = 0..T-2 of a correlator (host function of the
    library): "log" ln[C(y0)/C(y0+1)] or "cosh" (two-sided decay); NaN where
    undefined."""
    c = np.ascontiguousarray(cpp, dtype=np.float64)
    out = np.empty(max(len(c) - 1, 0), dtype=np.float64)
    _check(load().dp_effective_mass(c.ctypes.data, len(c), MEFF_KINDS[kind], out.ctypes.data))
    return out


def dp_fit_correlator(cpp, kind, t0, t1):
    """Least-squares fit of A exp(-m y0) ("log"/"exp") or A [exp(-m y0) +
    exp(-m (T - y0))] ("cosh") over y0 = t0..t1 in relative deviations;
    returns (m, A, rms relative deviation)."""
    c = np.ascontiguousarray(cpp, dtype=np.float64)
    m, A, rms = C.c_double(), C.c_double(), C.c_double()
    k = {"log": 0, "exp": 0, "cosh": 1}[kind]
    _check(load().dp_fit_correlator(c.ctypes.data, len(c), k, int(t0), int(t1), C.byref(m),
                                    C.byref(A), C.byref(rms)))
    return m.value, A.value, rms.value


def dp_solve_point_multi(ctx, field, Ms, profiles, src, r, opts=None, T=None, V=None,
                         want_prop=False, allow=(3,)):
    """Several masses (each with its profile) for one point source, one batch.

    Returns (cpp[n_mass, T], prop or None, [info dict per mass])."""
    n = len(Ms)
    Ma = np.ascontiguousarray(Ms, dtype=np.float64)
    profs = (Profile * n)()
    keep = []
    for k, p in enumerate(profiles):
        pr, kp = _profile(p)
        profs[k] = pr
        keep += kp
    cpp = np.zeros((n, int(T)))
    prop = np.zeros((n, 12, int(V), 4, 3), np.complex128) if want_prop else None
    infos = (SolveInfo * n)()
    o = _opts(opts)
    st = load().dp_solve_point_multi(ctx, int(field), n, _ptr(Ma), C.cast(profs, C.c_void_p),
                                     C.byref(_i4(src)), float(r), C.byref(o), _ptr(cpp),
                                     _ptr(prop) if want_prop else None, C.cast(infos, C.c_void_p))
    _check(st, allow)
    return cpp, prop, [i.as_dict() for i in infos]


def dp_solve_point_dev(ctx, field, Ms, profiles, src, r, cpp_out_dev, opts=None, allow=(3,)):
    """As dp_solve_point_multi with C_PP written to device memory at address
    `cpp_out_dev` (an int, e.g. a torch tensor's data_ptr()); returns infos."""
    n = len(Ms)
    Ma = np.ascontiguousarray(Ms, dtype=np.float64)
    profs = (Profile * n)()
    keep = []
    for k, p in enumerate(profiles):
        pr, kp = _profile(p)
        profs[k] = pr
        keep += kp
    infos = (SolveInfo * n)()
    o = _opts(opts)
    st = load().dp_solve_point_dev(ctx, int(field), n, _ptr(Ma), C.cast(profs, C.c_void_p),
                                   C.byref(_i4(src)), float(r), C.byref(o),
                                   C.c_void_p(int(cpp_out_dev)), C.cast(infos, C.c_void_p))
    _check(st, allow)
    return [i.as_dict() for i in infos]


# ---- operator application -------------------------------------------------------
def dp_apply(ctx, field, kind, M, profile, src, prec, psi, compress12=1):
    """out = op(psi) for host spinors (nrhs, T, Lz, Ly, Lx, 4, 3) complex128."""
    x = np.ascontiguousarray(psi, dtype=np.complex128)
    nrhs = x.shape[0]
    out = np.empty_like(x)
    pr, keep = _profile(profile)
    k = APPLY[kind] if isinstance(kind, str) else int(kind)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().dp_apply(ctx, int(field), k, float(M), C.byref(pr), C.byref(_i4(src or (0, 0, 0, 0))),
                           p, int(compress12), _ptr(x), _ptr(out), int(nrhs)))
    return out


def dp_profile_tables(dims, bc_t, profile, src=(0, 0, 0, 0)):
    """Host-side profile factors and hop coefficients: (alpha[4, Lmax], hop[4, 2, Lmax])."""
    Lm = max(int(d) for d in dims)
    alpha = np.zeros((4, Lm))
    hop = np.zeros((4, 2, Lm))
    pr, keep = _profile(profile)
    _check(load().dp_profile_tables(C.byref(_i4(dims)), int(bc_t), C.byref(pr), C.byref(_i4(src)),
                                    _ptr(alpha), _ptr(hop)))
    return alpha, hop


def pack_half_spinors(S, dims):
    """Host marshalling of lexicographic spinors S (n, T, Lz, Ly, Lx, 4, 3) into
    the packed even/odd device layout [12][V/2][n] (complex128): returns
    (even, odd) numpy arrays of shape (12, V/2, n)."""
    T, Lx, Ly, Lz = (int(d) for d in dims)
    S = np.asarray(S, dtype=np.complex128)
    n = S.shape[0]
    flat = S.reshape(n, T * Lz * Ly * Lx, 12)
    t, z, y, x = np.indices((T, Lz, Ly, Lx)).reshape(4, -1)
    par = (t + x + y + z) & 1
    idx = np.arange(T * Lz * Ly * Lx)
    out = []
    for p in (0, 1):
        sel = idx[par == p]
        half = sel >> 1
        a = np.zeros((12, T * Lx * Ly * Lz // 2, n), np.complex128)
        a[:, half, :] = flat[:, sel, :].transpose(2, 1, 0)
        out.append(a)
    return out[0], out[1]


def unpack_half_spinors(even, odd, dims):
    """Inverse of pack_half_spinors: (12, V/2, n) halves -> (n, T, Lz, Ly, Lx, 4, 3)."""
    T, Lx, Ly, Lz = (int(d) for d in dims)
    n = even.shape[2]
    V = T * Lz * Ly * Lx
    t, z, y, x = np.indices((T, Lz, Ly, Lx)).reshape(4, -1)
    par = (t + x + y + z) & 1
    idx = np.arange(V)
    flat = np.zeros((n, V, 12), np.complex128)
    for p, half in ((0, even), (1, odd)):
        sel = idx[par == p]
        flat[:, sel, :] = np.asarray(half)[:, sel >> 1, :].transpose(2, 1, 0)
    return flat.reshape(n, T, Lz, Ly, Lx, 4, 3)


def _groups(profiles, srcs):
    n = len(profiles)
    profs = (Profile * n)()
    keep = []
    for k, p in enumerate(profiles):
        pr, kp = _profile(p)
        profs[k] = pr
        keep += kp
    s = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32).reshape(n, 4))
    return n, profs, s, keep


def dp_restore_contract_dev(ctx, field, profiles, srcs, xe_ptr, xo_ptr, cpp_ptr):
    """Restore and contract device S' halves (packed layout) into device C_PP."""
    n, profs, s, keep = _groups(profiles, srcs)
    _check(load().dp_restore_contract_dev(ctx, int(field), n, C.cast(profs, C.c_void_p), _ptr(s),
                                          C.c_void_p(int(xe_ptr)), C.c_void_p(int(xo_ptr)),
                                          C.c_void_p(int(cpp_ptr))))


def dp_restore_contract_noalloc(ctx, field, profiles, srcs, xe_ptr, xo_ptr, cpp_ptr):
    """As dp_restore_contract_dev, with the device scratch in a fixed array
    inside the library: no device memory is allocated (see the header)."""
    n, profs, s, keep = _groups(profiles, srcs)
    _check(load().dp_restore_contract_noalloc(ctx, int(field), n, C.cast(profs, C.c_void_p),
                                              _ptr(s), C.c_void_p(int(xe_ptr)),
                                              C.c_void_p(int(xo_ptr)), C.c_void_p(int(cpp_ptr))))


def dp_spinor_bytes(ctx, field, prec, nrhs):
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    return int(load().dp_spinor_bytes(ctx, int(field), p, int(nrhs)))


def dp_dslash_dev(ctx, field, M, profile, prec, compress12, out_parity, in_ptr, out_ptr, nrhs,
                  block_threads=0, rhs_per_thread=0, iters=1, stages=-1):
    """Device-resident hopping application with the A^-1 epilogue; returns the
    average launch time in ms (CUDA events on the context stream)."""
    pr, keep = _profile(profile)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    ms = C.c_float()
    _check(load().dp_dslash_dev(ctx, int(field), float(M), C.byref(pr), p, int(compress12),
                                int(out_parity), C.c_void_p(int(in_ptr)), C.c_void_p(int(out_ptr)),
                                int(nrhs), int(block_threads), int(rhs_per_thread), int(stages),
                                int(iters), C.byref(ms)))
    return ms.value


def dp_schur_dev(ctx, field, M, profile, src, prec, compress12, parity, dagger, in_ptr, out_ptr,
                 nrhs):
    """out = Mhat in (dagger=0) or Mhat^dag in (dagger=1) on packed device
    spinors of one parity (the solvers' operators)."""
    pr, keep = _profile(profile)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    s = (C.c_int * 4)(*(src if src is not None else (0, 0, 0, 0)))
    _check(load().dp_schur_dev(ctx, int(field), float(M), C.byref(pr), C.byref(s), p,
                               int(compress12), int(parity), int(dagger), C.c_void_p(int(in_ptr)),
                               C.c_void_p(int(out_ptr)), int(nrhs)))


def dp_autotune(ctx, field, prec, compress12, nrhs):
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    b, rpt, sg, ms = C.c_int(), C.c_int(), C.c_int(), C.c_float()
    _check(load().dp_autotune(ctx, int(field), p, int(compress12), int(nrhs), C.byref(b),
                              C.byref(rpt), C.byref(sg), C.byref(ms)))
    return b.value, rpt.value, sg.value, ms.value


def dp_tune_set(ctx, field, prec, compress12, nrhs, block_threads, rhs_per_thread, stages):
    """Set the Schur dslash launch shape for this volume, precision and RHS
    count (e.g. from a tune cache) without timing."""
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check(load().dp_tune_set(ctx, int(field), p, int(compress12), int(nrhs), int(block_threads),
                              int(rhs_per_thread), int(stages)))


# ---- timing ----------------------------------------------------------------------
def dp_timing_enable(ctx, on=True):
    _check(load().dp_timing_enable(ctx, 1 if on else 0))


def dp_timing_reset(ctx):
    _check(load().dp_timing_reset(ctx))


def dp_timing_get(ctx, name):
    n, ms = C.c_long(), C.c_double()
    _check(load().dp_timing_get(ctx, name.encode(), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def dp_launch_count(ctx):
    return int(load().dp_launch_count(ctx))


# ---- serving -------------------------------------------------------------------------
def dp_serve_start(ctx, hbm_budget=0, max_slots=0):
    _check(load().dp_serve_start(ctx, int(hbm_budget), int(max_slots)))


def dp_submit(ctx, field, M, profile, src, r, prec="mixed_fp32", slice_tol=0.0):
    rq = Request()
    rq.field = int(field)
    rq.M = float(M)
    pr, keep = _profile(profile)
    rq.profile = pr
    rq.src = _i4(src)
    rq.r = float(r)
    rq.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    rq.slice_tol = float(slice_tol)
    t = C.c_uint64()
    _check(load().dp_submit(ctx, C.byref(rq), C.byref(t)))
    return t.value


def dp_wait(ctx, ticket, T, timeout_s=-1.0, allow=(3,)):
    cpp = np.zeros(int(T))
    info = SolveInfo()
    st = load().dp_wait(ctx, int(ticket), float(timeout_s), _ptr(cpp), C.byref(info))
    _check(st, allow)
    return cpp, info.as_dict()


def dp_cancel(ctx, ticket):
    _check(load().dp_cancel(ctx, int(ticket)))


def dp_serve_stats_get(ctx):
    s = ServeStats()
    _check(load().dp_serve_stats_get(ctx, C.byref(s)))
    return s.as_dict()


def dp_serve_stop(ctx, drain=True):
    _check(load().dp_serve_stop(ctx, 1 if drain else 0))
