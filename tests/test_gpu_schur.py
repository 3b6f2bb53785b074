"""The even-odd Schur operator Mhat and its adjoint (the operators of the
BiCGStab and CGNE solvers), through dp_schur_dev, against the oracle.

Mhat x = x - A_pp^-1 D_pq A_qq^-1 D_qp x is rebuilt here from the oracle's
full-lattice hopping term and clover term (A = 4 + M + clover inverted site by
site); the adjoint is checked through <u, Mhat v> = <Mhat^dag u, v>, which no
property of the implementation can fake.
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
import paper_1006_4028_gb300 as dp
from gpu_common import field, per_site_rel, require_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (8, 4, 6, 4)
M = 0.15
PROFILES = [(("none", 0.0), (0, 0, 0, 0)), (("cosh_t", 0.4), (3, 1, 2, 0)),
            (("exp_t", 0.3), (0, 0, 0, 0)), (("cosh_4d", 0.2), (5, 3, 0, 1))]


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    c = dp.dp_create(0)
    yield c
    dp.dp_destroy(c)


@pytest.fixture(scope="module")
def setup(ctx):
    U = field(DIMS, 0.5, 21)
    f = dp.dp_field_load(ctx, U, DIMS, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    op = oracle.WilsonClover(U, DIMS, 1.7, -1)
    # the site-local 12x12 matrix A = 4 + M + clover, column k = A e_k
    V = int(np.prod(DIMS))
    cols = []
    for k in range(12):
        e = np.zeros((1,) + oracle.array_shape(DIMS) + (4, 3), np.complex128)
        e[..., k // 3, k % 3] = 1
        cols.append(op.clover(e).reshape(V, 12))
    A = np.stack(cols, axis=-1) + (4 + M) * np.eye(12)
    return f, op, A


def ainv(A, psi):
    n = psi.shape[0]
    x = psi.reshape(n, -1, 12)
    y = np.linalg.solve(A[None], x[..., None])[..., 0]
    return y.reshape(psi.shape)


def parity_mask():
    t, z, y, x = np.indices(oracle.array_shape(DIMS))
    return ((t + x + y + z) % 2)


def oracle_mhat(op, A, v, p, prof, src):
    """v: full-lattice spinors supported on parity p."""
    par = parity_mask()
    pr = (prof[0], prof[1], src)
    t = op.hop(v, pr)
    t[:, par == p] = 0
    u = ainv(A, t)
    w = op.hop(u, pr)
    w[:, par != p] = 0
    out = v - ainv(A, w)
    out[:, par != p] = 0
    return out


def to_dev(half, prec):
    Vh = half.shape[1]
    if prec == "fp64":
        return torch.from_numpy(np.ascontiguousarray(half).view(np.float64)).cuda()
    n = half.shape[2]
    pr = half.reshape(12, Vh, n // 2, 2)
    b = np.stack([pr.real[..., 0], pr.real[..., 1], pr.imag[..., 0], pr.imag[..., 1]], -1)
    return torch.from_numpy(np.ascontiguousarray(b.astype(np.float32))).cuda()


def from_dev(t, prec, Vh, n):
    if prec == "fp64":
        return t.cpu().numpy().view(np.complex128).reshape(12, Vh, n)
    b = t.cpu().numpy().reshape(12, Vh, n // 2, 4).astype(np.float64)
    z = np.stack([b[..., 0] + 1j * b[..., 2], b[..., 1] + 1j * b[..., 3]], -1)
    return z.reshape(12, Vh, n)


def schur(ctx, f, prof, src, prec, p, dagger, half):
    n = half.shape[2]
    xin = to_dev(half, prec)
    out = torch.zeros_like(xin)
    dp.dp_schur_dev(ctx, f, M, prof, src, prec, 1, p, dagger, xin.data_ptr(), out.data_ptr(), n)
    torch.cuda.synchronize()
    return from_dev(out, prec, half.shape[1], n)


def half_of(psi, p):
    ev, od = dp.pack_half_spinors(psi, DIMS)
    return ev if p == 0 else od


def full_of(half, p):
    z = np.zeros_like(half)
    return dp.unpack_half_spinors(half, z, DIMS) if p == 0 else dp.unpack_half_spinors(z, half, DIMS)


@pytest.mark.parametrize("prof,src", PROFILES)
@pytest.mark.parametrize("p", [0, 1])
def test_mhat_fp64_matches_oracle(ctx, setup, prof, src, p):
    f, op, A = setup
    psi = li.random_spinor(DIMS, 4, 40 + p)
    h = half_of(psi, p)
    got = full_of(schur(ctx, f, prof, src, "fp64", p, 0, h), p)
    ref = oracle_mhat(op, A, full_of(h, p), p, prof, src)
    par = parity_mask()
    assert per_site_rel(got[:, par == p], ref[:, par == p]) < 1e-12


@pytest.mark.parametrize("prof,src", PROFILES)
@pytest.mark.parametrize("p", [0, 1])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed_fp32", 3e-6)])
def test_adjoint_identity(ctx, setup, prof, src, p, prec, tol):
    """<u, Mhat v> = <Mhat^dag u, v> per RHS; FP32 computes both sides in FP32."""
    f, op, A = setup
    u = half_of(li.random_spinor(DIMS, 4, 50 + p), p)
    v = half_of(li.random_spinor(DIMS, 4, 60 + p), p)
    mv = schur(ctx, f, prof, src, prec, p, 0, v)
    mdu = schur(ctx, f, prof, src, prec, p, 1, u)
    if prec != "fp64":  # the FP32 path sees FP32-rounded inputs
        u = u.astype(np.complex64).astype(np.complex128)
        v = v.astype(np.complex64).astype(np.complex128)
    lhs = np.einsum("csr,csr->r", np.conj(u), mv)
    rhs = np.einsum("csr,csr->r", np.conj(mdu), v)
    scale = np.linalg.norm(u.reshape(-1, 4), axis=0) * np.linalg.norm(mv.reshape(-1, 4), axis=0)
    assert np.max(np.abs(lhs - rhs) / scale) < tol
    # and the adjoint differs from the operator (the profile, gamma5 and the
    # clover placement all matter)
    assert np.max(np.abs(schur(ctx, f, prof, src, prec, p, 1, v) - mv)) > 1e-3


@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("prec,tol", [("mixed_fp32", 2e-6), ("mixed_fp16", 3e-3),
                                      ("mixed_bf16", 2e-2)])
def test_lower_precisions_track_fp64(ctx, setup, dagger, prec, tol):
    f, op, A = setup
    prof, src = PROFILES[3]
    h = half_of(li.random_spinor(DIMS, 6, 70), 1)
    ref = schur(ctx, f, prof, src, "fp64", 1, dagger, h)
    got = schur(ctx, f, prof, src, prec, 1, dagger, h)
    assert per_site_rel(np.moveaxis(got, 0, -1), np.moveaxis(ref, 0, -1)) < tol


def test_schur_bad_arguments(ctx, setup):
    f, _, _ = setup
    x = torch.zeros(16, device="cuda")
    for bad in [dict(parity=2), dict(dagger=3), dict(nrhs=0), dict(prec=9)]:
        a = dict(parity=0, dagger=0, nrhs=2, prec=1)
        a.update(bad)
        with pytest.raises(dp.DpError) as e:
            dp.dp_schur_dev(ctx, f, M, None, None, a["prec"], 1, a["parity"], a["dagger"],
                            x.data_ptr(), x.data_ptr() + 64, a["nrhs"])
        assert e.value.status == 1
    with pytest.raises(dp.DpError):  # odd nrhs in FP32
        dp.dp_schur_dev(ctx, f, M, None, None, "mixed_fp32", 1, 0, 0, x.data_ptr(),
                        x.data_ptr() + 64, 3)


# the launch shapes of the FP32 kernels the tuner chooses from (RHS per
# thread, staging, threads per block), 12-real and 18-real links
FUSED_SHAPES = [(1, 2, 6, 128), (1, 2, 6, 64), (1, 2, 0, 64), (1, 2, 2, 64), (1, 2, 5, 128),
                (0, 2, 6, 128), (0, 2, 0, 64)]


@pytest.mark.parametrize("c12,rpt,stages,block", FUSED_SHAPES)
def test_fused_ainv_dslash_per_site(ctx, setup, c12, rpt, stages, block):
    """The benchmark's launch A_ee^-1 D_eo psi_o (FP32, fused clover-inverse
    epilogue) directly against the oracle: its hopping term on the odd-parity
    input, then the inverse of the site matrix A = 4 + M + clover, per site
    and right-hand side at 1e-6 (the oracle takes the FP32-rounded input)."""
    f, op, A = setup
    prof = ("cosh_4d", 0.3)
    psi = li.random_spinor(DIMS, 12, 81).astype(np.complex64).astype(np.complex128)
    ev, od = dp.pack_half_spinors(psi, DIMS)
    xin = to_dev(od, "mixed_fp32")
    out = torch.zeros_like(xin)
    dp.dp_dslash_dev(ctx, f, M, prof, "mixed_fp32", c12, 0, xin.data_ptr(), out.data_ptr(), 12,
                     block, rpt, 1, stages=stages)
    torch.cuda.synchronize()
    got = full_of(from_dev(out, "mixed_fp32", ev.shape[1], 12), 0)
    par = parity_mask()
    t = op.hop(full_of(od, 1), (prof[0], prof[1], (0, 0, 0, 0)))
    t[:, par != 0] = 0
    ref = ainv(A, t)
    assert per_site_rel(got[:, par == 0], ref[:, par == 0]) < 1e-6


@pytest.mark.parametrize("prof,src", PROFILES)
@pytest.mark.parametrize("p", [0, 1])
def test_mhat_fp32_per_site(ctx, setup, prof, src, p):
    """Mhat in FP32 (its second launch is the fused x - A^-1 D epilogue) per
    site against the oracle's Schur complement at 1e-6."""
    f, op, A = setup
    psi = li.random_spinor(DIMS, 12, 90 + p).astype(np.complex64).astype(np.complex128)
    h = half_of(psi, p)
    got = full_of(schur(ctx, f, prof, src, "mixed_fp32", p, 0, h), p)
    ref = oracle_mhat(op, A, full_of(h, p), p, prof, src)
    par = parity_mask()
    assert per_site_rel(got[:, par == p], ref[:, par == p]) < 1e-6
