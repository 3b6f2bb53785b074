"""CPU oracle for distance-preconditioned Wilson-clover solves (arXiv 1006.4028).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the GPU library never does, and
this package never imports the GPU library.  It shares no code with it; the
two meet only in the seeded input generators of ``lattice_inputs``.

Plain FP64, full lattice (no even-odd split), lexicographic sites, explicit
4x4 gamma matrices and uncompressed links.  The heavy loops live in
``dirac.c`` (plain C, OpenMP over sites); this module holds the conventions,
the preconditioning profiles, the point-source pipeline (source scaling,
solve, restore, contraction) and the closed forms the oracle is pinned to.

Profile orientation.  The paper (Sec. II, eq. redeft) writes S = alpha S'.
The library and this oracle take the reciprocal profile alpha_B = 1/alpha:
S' = alpha_B S and eta' = alpha_B eta, so that the preconditioned operator is
A (D+M) A^-1 with A = diag(alpha_B).  In that orientation the coefficient of
U_mu(x) psi'(x+mu) is alpha_B(x_mu)/alpha_B(x_mu+1) (Sec. II modified forward
derivative, eq. redefcovs for all directions) and the profiles read

* ``cosh_t``  alpha_B = 1/cosh[alpha0 (y0 - T/2)]          (eq. pbcalpha)
* ``exp_t``   alpha_B = exp(+alpha0 y0)                     (Sec. II, SF form)
* ``cosh_4d`` alpha_B = prod_mu cosh[alpha0 (y_mu - L_mu/2)] (eq. betaa)

with every coordinate taken relative to the source, (y - x_src) mod L.  The
boundary sign (antiperiodic time) stays on the absolute seam t = T-1 -> 0,
where the hop factor is the ratio of the two sites' profile values times the
sign: this is eq. (redeftbc).

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_*.py`` (closed forms, dense LU, symmetries).  The
effective masses and the correlator fit (the paper plots effective masses
without writing a definition out; the log-ratio and cosh readings) are
pinned to exact one- and two-sided exponentials and to the free-theory pole
2 ln(1+M) of the pseudoscalar at zero momentum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile ``dirac.c`` into ``_build/liboracle.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "dirac.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    )
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.or_hop.argtypes = [vp, vp, vp, vp, vp, ip, vp, vp, ip]
            lib.or_field_strength.argtypes = [vp, vp, vp]
            lib.or_clover.argtypes = [vp, vp, vp, dp, vp, vp, ip]
            lib.or_clover_matrix.argtypes = [vp, vp, vp, dp, vp]
            lib.or_dirac.argtypes = [vp, vp, vp, vp, dp, vp, vp, ip, vp, vp, ip]
            lib.or_bicgstab.argtypes = [vp, vp, vp, vp, dp, vp, vp, ip, vp, vp,
                                        ip, dp, ip, vp, vp]
            lib.or_bicgstab.restype = ip
            lib.or_num_threads.restype = ip
            _lib = lib
    return _lib


def num_threads():
    """Host threads the oracle's OpenMP loops use."""
    return int(_load().or_num_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


# --------------------------------------------------------------------------
# Dirac algebra (chiral basis; the paper does not fix a basis)
# --------------------------------------------------------------------------
def gammas():
    """Euclidean gamma_0..gamma_3 in the chiral basis, shape (4, 4, 4).

    gamma_mu = [[0, e_mu], [e_mu^dag, 0]] with e_0 = -1 and e_k = -i sigma_k,
    so that gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1, 1, -1, -1).
    """
    s = [np.array([[0, 1], [1, 0]], complex),
         np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex)]
    e = [-np.eye(2, dtype=complex)] + [-1j * sk for sk in s]
    g = np.zeros((4, 4, 4), complex)
    for mu in range(4):
        g[mu, :2, 2:] = e[mu]
        g[mu, 2:, :2] = e[mu].conj().T
    return g


def gamma5():
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def sigmas():
    """sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], shape (4, 4, 4, 4)."""
    g = gammas()
    sg = np.zeros((4, 4, 4, 4), complex)
    for mu in range(4):
        for nu in range(4):
            sg[mu, nu] = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
    return sg


# --------------------------------------------------------------------------
# Geometry helpers
# --------------------------------------------------------------------------
def dims_tuple(dims):
    return tuple(int(d) for d in dims)


def volume(dims):
    T, Lx, Ly, Lz = dims_tuple(dims)
    return T * Lx * Ly * Lz


def array_shape(dims):
    T, Lx, Ly, Lz = dims_tuple(dims)
    return (T, Lz, Ly, Lx)


_AXIS = {0: 0, 1: 3, 2: 2, 3: 1}  # direction mu -> axis of a (T, Lz, Ly, Lx) array


def site_coords(dims):
    """Coordinates (t, x, y, z) of every site, each of shape (T, Lz, Ly, Lx)."""
    c = np.indices(array_shape(dims))
    return [c[_AXIS[mu]] for mu in range(4)]


# --------------------------------------------------------------------------
# Preconditioning profiles (alpha_B orientation, see module docstring)
# --------------------------------------------------------------------------
PROFILE_KINDS = ("none", "exp_t", "cosh_t", "cosh_4d", "table")


def profile_alpha(kind, alpha0, dims, src=(0, 0, 0, 0), tables=None):
    """Per-direction profile factors alpha_B,mu(x_mu), a list of 4 arrays.

    The site profile is alpha_B(x) = prod_mu alpha_B,mu(x_mu).  Coordinates
    enter relative to the source, (x_mu - src_mu) mod L_mu.
    """
    d = dims_tuple(dims)
    out = []
    for mu in range(4):
        L = d[mu]
        rel = (np.arange(L) - int(src[mu])) % L
        if kind == "none":
            a = np.ones(L)
        elif kind == "exp_t":
            a = np.exp(alpha0 * rel) if mu == 0 else np.ones(L)
        elif kind == "cosh_t":
            a = 1.0 / np.cosh(alpha0 * (rel - L / 2.0)) if mu == 0 else np.ones(L)
        elif kind == "cosh_4d":
            a = np.cosh(alpha0 * (rel - L / 2.0))
        elif kind == "table":
            a = np.asarray(tables[mu], dtype=np.float64).copy()
            assert a.shape == (L,)
        else:
            raise ValueError(kind)
        out.append(np.asarray(a, dtype=np.float64))
    return out


def site_alpha(alphas, dims):
    """alpha_B(x) = prod_mu alpha_B,mu(x_mu) on the lattice, shape (T, Lz, Ly, Lx)."""
    c = site_coords(dims)
    a = np.ones(array_shape(dims))
    for mu in range(4):
        a = a * alphas[mu][c[mu]]
    return a


def hop_tables(alphas, dims, bc_t):
    """Forward/backward hop coefficients per direction and coordinate.

    fwd[mu][x] multiplies U_mu(x) psi(x+mu):   alpha_B(x)/alpha_B(x+1)
    bwd[mu][x] multiplies U_mu(x-mu)^dag psi(x-mu): alpha_B(x)/alpha_B(x-1)
    (the paper's modified derivatives, Sec. II and eq. redefcovs, in the
    alpha_B = 1/alpha orientation), with the time boundary sign bc_t on the
    hops that cross t = T-1 <-> 0 (eq. redeftbc).
    """
    d = dims_tuple(dims)
    ldt = max(d)
    fwd = np.zeros((4, ldt))
    bwd = np.zeros((4, ldt))
    for mu in range(4):
        L = d[mu]
        a = alphas[mu]
        for x in range(L):
            xp, xm = (x + 1) % L, (x - 1) % L
            sf = bc_t if (mu == 0 and x == L - 1) else 1.0
            sb = bc_t if (mu == 0 and x == 0) else 1.0
            fwd[mu, x] = sf * a[x] / a[xp]
            bwd[mu, x] = sb * a[x] / a[xm]
    return fwd, bwd, ldt


# --------------------------------------------------------------------------
# Operator
# --------------------------------------------------------------------------
class WilsonClover:
    """(D'[U] + M) on the full lattice; see ``dirac.c`` for the formula.

    links: complex128 (T, Lz, Ly, Lx, 4, 3, 3); dims = (T, Lx, Ly, Lz);
    bc_t = -1 for antiperiodic time, +1 for periodic; space is periodic.
    """

    def __init__(self, links, dims, csw, bc_t=-1):
        self.dims = dims_tuple(dims)
        self.d = np.array(self.dims, dtype=np.int32)
        self.V = volume(dims)
        self.U = _c128(links).reshape(self.V, 4, 3, 3)
        self.csw = float(csw)
        self.bc_t = float(bc_t)
        self.gam = _c128(gammas())
        self.sig = _c128(sigmas())
        self.F = np.zeros((self.V, 4, 4, 3, 3), np.complex128)
        _load().or_field_strength(_p(self.d), _p(self.U), _p(self.F))
        # the clover term as one 12x12 matrix per site (same definition)
        self.Cm = None
        if self.csw != 0.0:
            self.Cm = np.zeros((self.V, 12, 12), np.complex128)
            _load().or_clover_matrix(_p(self.d), _p(self.F), _p(self.sig), self.csw, _p(self.Cm))

    def _cm(self):
        return _p(self.Cm) if self.Cm is not None else None

    def tables(self, profile=None):
        if profile is None:
            profile = ("none", 0.0, (0, 0, 0, 0))
        kind, alpha0, src = profile[:3]
        tabs = profile[3] if len(profile) > 3 else None
        al = profile_alpha(kind, alpha0, self.dims, src, tabs)
        fwd, bwd, ldt = hop_tables(al, self.dims, self.bc_t)
        return np.ascontiguousarray(fwd), np.ascontiguousarray(bwd), ldt, al

    def _spin(self, psi):
        psi = _c128(psi)
        n = psi.size // (self.V * 12)
        assert psi.size == n * self.V * 12
        return psi, n

    def hop(self, psi, profile=None):
        psi, n = self._spin(psi)
        fwd, bwd, ldt, _ = self.tables(profile)
        out = np.empty_like(psi)
        _load().or_hop(_p(self.d), _p(self.U), _p(self.gam), _p(fwd), _p(bwd), ldt,
                       _p(psi), _p(out), n)
        return out

    def clover(self, psi):
        psi, n = self._spin(psi)
        out = np.empty_like(psi)
        _load().or_clover(_p(self.d), _p(self.F), _p(self.sig), self.csw, _p(psi), _p(out), n)
        return out

    def apply(self, psi, M, profile=None):
        psi, n = self._spin(psi)
        fwd, bwd, ldt, _ = self.tables(profile)
        out = np.empty_like(psi)
        _load().or_dirac(_p(self.d), _p(self.U), self._cm(), _p(self.gam), float(M), _p(fwd),
                         _p(bwd), ldt, _p(psi), _p(out), n)
        return out

    def solve(self, b, M, profile=None, tol=1e-13, maxit=20000, x0=None):
        """BiCGStab on the full lattice; returns (x, iters[n], relres[n], ok)."""
        b, n = self._spin(b)
        fwd, bwd, ldt, _ = self.tables(profile)
        x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
        iters = np.zeros(n, np.int32)
        rel = np.zeros(n)
        st = _load().or_bicgstab(_p(self.d), _p(self.U), self._cm(), _p(self.gam), float(M),
                                 _p(fwd), _p(bwd), ldt, _p(b), _p(x), n, float(tol), int(maxit),
                                 _p(iters), _p(rel))
        return x, iters, rel, st == 0


# --------------------------------------------------------------------------
# Point-source pipeline: source scaling, solve, restore, contract
# --------------------------------------------------------------------------
def point_sources(dims, src, scale=1.0):
    """The 12 spin-colour point sources at ``src = (t, x, y, z)``, times ``scale``.

    Returns complex128 (12, T, Lz, Ly, Lx, 4, 3); RHS k = 3*spin + colour.
    """
    eta = np.zeros((12,) + array_shape(dims) + (4, 3), np.complex128)
    t, x, y, z = (int(v) for v in src)
    for k in range(12):
        eta[k, t, z, y, x, k // 3, k % 3] = scale
    return eta


def restore(Sp, alphas, dims):
    """S(y) = S'(y) / alpha_B(y), per site (Sec. II eq. redeft; Sec. III eq. redefa)."""
    a = site_alpha(alphas, dims)
    shp = (1,) + array_shape(dims) + (1, 1)
    return Sp / a.reshape(shp)


def contract_cpp(S, dims, t_src):
    """C_PP(y0) = -sum_{y vec} tr[S^dag S] (Sec. II), y0 relative to t_src.

    S: (12, T, Lz, Ly, Lx, 4, 3) solutions for the 12 source components.
    """
    T = dims_tuple(dims)[0]
    per_t = np.sum(np.abs(S) ** 2, axis=(0, 2, 3, 4, 5, 6))
    return -np.roll(per_t, -int(t_src))


def contract_cap(S, dims, t_src):
    """C_AP(y0) = sum_{y vec} tr[gamma_0 S S^dag], y0 relative to t_src.

    The axial-pseudoscalar correlator of the pair of degenerate quarks whose
    pseudoscalar correlator is C_PP: with S(x, y) = gamma_5 S(y, x)^dag
    gamma_5, -tr[gamma_0 gamma_5 S(y,x) gamma_5 S(x,y)] = tr[gamma_0 S S^dag]
    (gamma_5 gamma_0 gamma_5 = -gamma_0); same orientation and normalisation as
    contract_cpp.  S: (12, T, Lz, Ly, Lx, 4, 3).
    """
    g0 = _c128(gammas()[0])
    # tr[gamma_0 S S^dag] = sum_{j, c, s1, s2} g0[s1, s2] S_j(s2, c) conj(S_j(s1, c))
    per_t = np.einsum("ab,jtzyxbc,jtzyxac->t", g0, S, np.conj(S)).real
    return np.roll(per_t, -int(t_src))


def contract_hl(Sh, Sl, dims, t_src):
    """Heavy-light pseudoscalar correlator C(y0) = -sum_{y vec} tr[S_h S_l^dag]
    (= -tr[gamma_5 S_h(y,x) gamma_5 S_l(x,y)] by gamma_5-hermiticity), complex,
    y0 relative to t_src.  Sh, Sl: (12, T, Lz, Ly, Lx, 4, 3), each restored by
    its own profile (Sec. III: restore before contracting)."""
    per_t = np.einsum("jtzyxsc,jtzyxsc->t", Sh, np.conj(Sl))
    return -np.roll(per_t, -int(t_src))


def pcac_mass(cpp, cap):
    """m_PCAC(y0) = [C_AP(y0+1) - C_AP(y0-1)] / 2 / (2 C_PP(y0)), y0 = 1..T-2
    (the unimproved local-current ratio; the paper quotes am_PCAC to label its
    quark masses, Sec. II).  Returns an array of length T, NaN at the ends."""
    cpp = np.asarray(cpp, float)
    cap = np.asarray(cap, float)
    m = np.full(len(cpp), np.nan)
    m[1:-1] = (cap[2:] - cap[:-2]) / 2.0 / (2.0 * cpp[1:-1])
    return m


def solve_point(op, M, profile_kind="none", alpha0=0.0, src=(0, 0, 0, 0), tol=1e-13,
                maxit=20000, tables=None):
    """Full method for a point source: eta' = alpha_B(x_src) eta, solve
    (D'+M) S' = eta', restore S = S'/alpha_B, contract C_PP.

    Returns (cpp[T], S restored, info dict).
    """
    dims = op.dims
    prof = (profile_kind, alpha0, tuple(src), tables)
    al = profile_alpha(profile_kind, alpha0, dims, src, tables)
    a_src = 1.0
    for mu in range(4):
        a_src *= al[mu][int(src[mu])]
    eta_p = point_sources(dims, src, a_src)
    Sp, iters, rel, ok = op.solve(eta_p, M, prof, tol=tol, maxit=maxit)
    S = restore(Sp, al, dims)
    cpp = contract_cpp(S, dims, src[0])
    return cpp, S, {"iters": iters, "relres": rel, "converged": ok, "Sprime": Sp,
                    "cap": contract_cap(S, dims, src[0])}


def slice_residuals(op, M, S, eta, t_src=0):
    """Per-time-slice relative residual of a restored solution.

    rho(y0) = |[eta - (D+M) S]_t| / |S_t| with |.|_t the L2 norm over the
    spatial sites of time slice t = (y0 + t_src) mod T and over all right-hand
    sides (the 12 components of a point source), on the unpreconditioned
    system of Sec. I eq. (linsysunprec).  The paper's global criterion (eq.
    stopping) bounds only the sum over slices; this is the quantity whose
    smallness on the far slices decides whether C_PP(y0) is accurate there
    (Sec. II, the error argument behind the preconditioning).
    S, eta: (n, T, Lz, Ly, Lx, 4, 3).  Returns an array of length T.
    """
    S = _c128(S)
    r = _c128(eta) - op.apply(S, M)
    T = dims_tuple(op.dims)[0]
    n = S.size // (op.V * 12)
    rt = np.sum(np.abs(r.reshape(n, T, -1)) ** 2, axis=(0, 2))
    st = np.sum(np.abs(S.reshape(n, T, -1)) ** 2, axis=(0, 2))
    return np.roll(np.sqrt(rt / st), -int(t_src))


def effective_mass(cpp):
    """m_eff(y0) = ln[C(y0)/C(y0+1)] (log-ratio reading; the paper plots it
    without writing it out)."""
    c = np.asarray(cpp)
    return np.log(c[:-1] / c[1:])


def _log_cosh(x):
    x = np.abs(x)
    return x + np.log1p(np.exp(-2.0 * x)) - np.log(2.0)


def effective_mass_cosh(cpp):
    """Cosh-form effective mass on a lattice with two-sided decay: m(y0) > 0
    with C(y0)/C(y0+1) = cosh[m (T/2 - y0)] / cosh[m (T/2 - y0 - 1)] (a state
    propagating both ways round the periodic time direction).  NaN where the
    ratio has no such solution.  Root by Brent's method."""
    from scipy.optimize import brentq

    c = np.asarray(cpp, dtype=float)
    T = len(c)
    out = np.full(T - 1, np.nan)
    for t in range(T - 1):
        r = c[t] / c[t + 1]
        if not (r > 0 and np.isfinite(r)):
            continue
        a, b = T / 2.0 - t, T / 2.0 - t - 1.0

        def f(m):
            return _log_cosh(m * a) - _log_cosh(m * b) - np.log(r)

        lo, hi = 1e-12, 50.0
        if f(lo) * f(hi) < 0:
            out[t] = brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    return out


def fit_correlator(cpp, kind, t0, t1):
    """Least-squares fit of C(y0) = A exp(-m y0) (kind "exp") or
    A [exp(-m y0) + exp(-m (T - y0))] (kind "cosh") to y0 = t0..t1, in the
    relative deviations A model/C - 1 (no statistical weights: one synthetic
    configuration).  Both parameters by scipy's trust-region least squares
    from the log-ratio effective mass at the window's start.  Returns
    (m, A, rms relative deviation)."""
    from scipy.optimize import least_squares

    c = np.asarray(cpp, dtype=float)
    T = len(c)
    t = np.arange(t0, t1 + 1, dtype=float)
    ct = c[t0:t1 + 1]

    def model(m):
        f = np.exp(-m * t)
        if kind == "cosh":
            f = f + np.exp(-m * (T - t))
        return f

    m0 = max(np.log(c[t0] / c[t0 + 1]), 1e-3)
    A0 = ct[0] / model(m0)[0]
    res = least_squares(lambda p: p[0] * model(p[1]) / ct - 1.0, x0=[A0, m0], xtol=1e-15,
                        ftol=1e-15, gtol=1e-15, method="lm")
    A, m = res.x
    dev = A * model(m) / ct - 1.0
    return float(m), float(A), float(np.sqrt(np.mean(dev ** 2)))


# --------------------------------------------------------------------------
# Closed forms used as pins
# --------------------------------------------------------------------------
def free_momentum_operator(p, M):
    """D(p) = M + sum_mu [i gamma_mu sin p_mu + 1 - cos p_mu] (4x4), free Wilson."""
    g = gammas()
    D = M * np.eye(4, dtype=complex)
    for mu in range(4):
        D = D + 1j * g[mu] * np.sin(p[mu]) + (1 - np.cos(p[mu])) * np.eye(4)
    return D


def free_propagator(dims, M, bc_t=-1):
    """Exact free Wilson propagator from the origin, by momentum sums.

    S(x) = (1/V) sum_p e^{i p.x} D(p)^-1 with p_mu = 2 pi n_mu / L_mu and, for
    antiperiodic time, p_0 = 2 pi (n_0 + 1/2)/T.  Returns (T, Lz, Ly, Lx, 4, 4)
    (colour is the identity).
    """
    T, Lx, Ly, Lz = dims_tuple(dims)
    shp = (T, Lz, Ly, Lx)
    shift0 = 0.5 if bc_t < 0 else 0.0
    n = np.indices(shp)
    p = [2 * np.pi * (n[0] + shift0) / T, 2 * np.pi * n[3] / Lx,
         2 * np.pi * n[2] / Ly, 2 * np.pi * n[1] / Lz]
    g = gammas()
    m = M + sum(1 - np.cos(pm) for pm in p)
    den = sum(np.sin(pm) ** 2 for pm in p) + m ** 2
    num = np.zeros(shp + (4, 4), complex)
    for mu in range(4):
        num -= 1j * np.sin(p[mu])[..., None, None] * g[mu]
    num += m[..., None, None] * np.eye(4)
    Dinv = num / den[..., None, None]
    S = np.fft.ifftn(Dinv, axes=(0, 1, 2, 3))
    t = np.arange(T).reshape(T, 1, 1, 1, 1, 1)
    return S * np.exp(1j * np.pi * shift0 * 2 * t / T)


def free_cpp(dims, M, bc_t=-1):
    """C_PP(y0) of the exact free propagator (3 colours, all 4x4 spin entries)."""
    S = free_propagator(dims, M, bc_t)
    return -3.0 * np.sum(np.abs(S) ** 2, axis=(1, 2, 3, 4, 5))


def dense_matrix(op, M, profile=None, batch=768):
    """(D'+M) as a dense (12V, 12V) matrix, built column by column from unit vectors."""
    N = op.V * 12
    A = np.zeros((N, N), np.complex128)
    for j0 in range(0, N, batch):
        nb = min(batch, N - j0)
        E = np.zeros((nb, N), np.complex128)
        E[np.arange(nb), j0 + np.arange(nb)] = 1
        A[:, j0:j0 + nb] = op.apply(E, M, profile).reshape(nb, N).T
    return A


# --------------------------------------------------------------------------
# 16-bit link storage (the compressed gauge field of the mixed-precision
# inner solver): what the operator sees when the links are kept as rows 0
# and 1 in FP16 or BF16 with one FP32 scale per link and row 2 rebuilt.
# --------------------------------------------------------------------------
def round_bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32.

    bfloat16 is the upper 16 bits of an IEEE float32; rounding adds half an
    ulp of the kept part (0x7FFF, plus the kept part's last bit for ties) to
    the 32-bit pattern and clears the low 16 bits.  Finite inputs only.
    """
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def stored_links16(links, kind):
    """The gauge field as the 16-bit storage reproduces it, in FP64.

    Per link U: s = fp32(max of |Re|, |Im| over rows 0 and 1) (1 if that is
    0); each of those 12 reals r is kept as q = round16(fp32(r * (1/s))) with
    round16 = FP16 or BF16 round-to-nearest-even; the operator uses s*q for
    rows 0 and 1 and row 2 = conj(row0 x row1), which is the third row of a
    special unitary matrix (the SU(3) links of Sec. I).  kind: "fp16" | "bf16".
    """
    U = _c128(links)
    rows = U[..., :2, :]
    re, im = rows.real, rows.imag
    mx = np.maximum(np.abs(re), np.abs(im)).max(axis=(-2, -1))
    s = mx.astype(np.float32)
    s = np.where(s > 0, s, np.float32(1.0)).astype(np.float64)
    inv = (1.0 / s)[..., None, None]

    def q(a):
        a32 = (a * inv).astype(np.float32)
        if kind == "fp16":
            return a32.astype(np.float16).astype(np.float64)
        if kind == "bf16":
            return round_bf16(a32).astype(np.float64)
        raise ValueError("kind must be 'fp16' or 'bf16'")

    r01 = (q(re) + 1j * q(im)) * s[..., None, None]
    out = np.empty_like(U)
    out[..., :2, :] = r01
    out[..., 2, :] = np.conj(np.cross(r01[..., 0, :], r01[..., 1, :]))
    return out
