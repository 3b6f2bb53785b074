"""GPU parity of the operator kernels against the CPU oracle, through the C ABI.

Tolerances (per site, |GPU(x) - oracle(x)|_2 / |oracle(x)|_2, max over sites):
FP64 1e-13, FP32 1e-6 (the FP32 path is fed the FP32-rounded spinor and links,
the oracle the FP64 ones).
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
import paper_1006_4028_gb300 as dp
from gpu_common import field, per_site_rel, require_gpu

pytestmark = pytest.mark.gpu

PROFILES = [("none", 0.0, (0, 0, 0, 0)), ("cosh_t", 0.4, (3, 1, 2, 0)),
            ("exp_t", 0.4, (0, 0, 0, 0)), ("cosh_4d", 0.2, (5, 3, 0, 1))]


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    c = dp.dp_create(0)
    yield c
    dp.dp_destroy(c)


@pytest.fixture(scope="module")
def setup(ctx):
    dims = (8, 4, 6, 4)
    U = field(dims, 0.5, 11)
    f = dp.dp_field_load(ctx, U, dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    op = oracle.WilsonClover(U, dims, 1.7, -1)
    psi = li.random_spinor(dims, 3, 12)
    return dims, f, op, psi


@pytest.mark.parametrize("prof", PROFILES)
def test_hop_fp64(ctx, setup, prof):
    dims, f, op, psi = setup
    kind, a0, src = prof
    got = dp.dp_apply(ctx, f, "hop", 0.0, (kind, a0), src, "fp64", psi)
    ref = op.hop(psi, (kind, a0, src))
    assert per_site_rel(got, ref) < 1e-13


@pytest.mark.parametrize("prof", PROFILES)
@pytest.mark.parametrize("c12", [0, 1])
def test_hop_fp32(ctx, setup, prof, c12):
    dims, f, op, psi = setup
    kind, a0, src = prof
    got = dp.dp_apply(ctx, f, "hop", 0.0, (kind, a0), src, "mixed_fp32", psi, compress12=c12)
    ref = op.hop(psi, (kind, a0, src))
    assert per_site_rel(got, ref) < 1e-6


@pytest.mark.parametrize("prof", PROFILES)
@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_hop_16bit_links(ctx, setup, prof, kind):
    """16-bit links: the FP32 kernel against the oracle run on the links as
    the 16-bit storage reproduces them (quantised rows 0, 1; row 2 rebuilt)."""
    dims, f, op, psi = setup
    kp, a0, src = prof
    got = dp.dp_apply(ctx, f, "hop", 0.0, (kp, a0), src, "mixed_" + kind, psi)
    op16 = oracle.WilsonClover(oracle.stored_links16(op.U.reshape(oracle.array_shape(dims) + (4, 3, 3)),
                                                     kind), dims, 0.0, -1)
    assert per_site_rel(got, op16.hop(psi, (kp, a0, src))) < 1e-6
    # and the quantisation is visible against the unquantised links
    err = per_site_rel(got, op.hop(psi, (kp, a0, src)))
    assert 1e-5 < err < (2e-2 if kind == "bf16" else 3e-3)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed_fp32", 1e-6)])
def test_clover_and_full_operator(ctx, setup, prec, tol):
    dims, f, op, psi = setup
    got = dp.dp_apply(ctx, f, "clover", 0.0, None, None, prec, psi)
    assert per_site_rel(got, op.clover(psi)) < tol
    M = 0.3
    prof = ("cosh_4d", 0.3, (1, 2, 3, 0))
    got = dp.dp_apply(ctx, f, "full", M, prof[:2], prof[2], prec, psi)
    assert per_site_rel(got, op.apply(psi, M, prof)) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed_fp32", 2e-6)])
def test_clover_inverse(ctx, setup, prec, tol):
    dims, f, op, psi = setup
    M = 0.05
    y = dp.dp_apply(ctx, f, "clover_inv", M, None, None, prec, psi)
    back = (4 + M) * y + op.clover(y)
    assert per_site_rel(back, psi) < tol


def test_free_field_clover_vanishes_and_unit_links(ctx):
    dims = (4, 4, 4, 4)
    U = li.unit_links(dims)
    f = dp.dp_field_load(ctx, U, dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.9)
    psi = li.random_spinor(dims, 1, 3)
    assert np.abs(dp.dp_apply(ctx, f, "clover", 0.0, None, None, "fp64", psi)).max() == 0.0
    op = oracle.WilsonClover(U, dims, 1.9, -1)
    got = dp.dp_apply(ctx, f, "full", 0.5, None, None, "fp64", psi)
    assert per_site_rel(got, op.apply(psi, 0.5)) < 1e-13
    dp.dp_field_free(ctx, f)


def test_periodic_time_and_many_rhs(ctx):
    dims = (4, 6, 4, 2)
    U = field(dims, 0.3, 5)
    f = dp.dp_field_load(ctx, U, dims, +1)
    dp.dp_field_set_csw(ctx, f, 1.0)
    op = oracle.WilsonClover(U, dims, 1.0, +1)
    psi = li.random_spinor(dims, 13, 6)  # ragged: 13 RHS
    got = dp.dp_apply(ctx, f, "full", 0.1, ("exp_t", 0.3), (1, 0, 0, 0), "fp64", psi)
    assert per_site_rel(got, op.apply(psi, 0.1, ("exp_t", 0.3, (1, 0, 0, 0)))) < 1e-13
    dp.dp_field_free(ctx, f)


def test_invalid_arguments_are_errors(ctx):
    dims = (4, 4, 4, 4)
    U = li.unit_links(dims)
    with pytest.raises(dp.DpError) as e:  # odd extent: no even-odd split
        dp.dp_field_load(ctx, li.unit_links((4, 3, 4, 4)), (4, 3, 4, 4), -1)
    assert e.value.status == 1
    with pytest.raises(dp.DpError) as e:  # bc_t must be -1, 0 (Dirichlet) or +1
        dp.dp_field_load(ctx, U, dims, 2)
    assert e.value.status == 1
    bad = U.copy()
    bad[0, 0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(dp.DpError) as e:
        dp.dp_field_load(ctx, bad, dims, -1)
    assert e.value.status == 1
    with pytest.raises(dp.DpError) as e:
        dp.dp_field_set_csw(ctx, 987654, 1.0)
    assert e.value.status == 9
    f = dp.dp_field_load(ctx, U, dims, -1)
    psi = li.random_spinor(dims, 1, 1)
    with pytest.raises(dp.DpError):  # clover not built yet
        dp.dp_apply(ctx, f, "full", 0.1, None, None, "fp64", psi)
    psi[0, 0, 0, 0, 0, 0, 0] = np.inf
    with pytest.raises(dp.DpError):
        dp.dp_apply(ctx, f, "hop", 0.1, None, None, "fp64", psi)
    dp.dp_field_free(ctx, f)
    with pytest.raises(dp.DpError):
        dp.dp_field_free(ctx, f)


# (RHS per thread, shared-memory stages, threads per block); 96, 128 and 160
# threads leave a ragged last block on the 8x4x6x4 lattice (2304 pairs)
SHAPES32 = [(2, 0, 64), (4, 0, 64), (2, 2, 64), (2, 3, 128), (2, 3, 96), (2, 2, 96),
            (4, 0, 256), (2, 0, 160), (2, 4, 64), (2, 4, 96), (2, 4, 128), (2, 5, 64),
            (2, 5, 160), (2, 5, 128), (2, 5, 256), (2, 6, 64), (2, 6, 96), (2, 6, 128)]


# 18-real FP32 links: the direct kernels and the spinor-staged one
SHAPES32_18 = [(2, 0, 64), (2, 6, 64), (2, 6, 96), (2, 6, 128), (4, 0, 64)]


@pytest.mark.parametrize("prec,tol,rpts,c12", [("mixed_fp32", 1e-6, SHAPES32, 1),
                                               ("mixed_fp32", 1e-6, SHAPES32_18, 0),
                                               ("fp64", 1e-13, [(1, 0, 64), (1, 0, 160)], 1)])
def test_schur_launch_all_rhs_per_thread(ctx, setup, prec, tol, rpts, c12):
    """out_e = A_ee^-1 D_eo psi_o on packed device spinors (the solver's launch),
    for every launch shape (RHS per thread, staging, block): bit-identical to
    each other and, through A_ee out_e = D_eo psi_o, equal to the oracle."""
    torch = pytest.importorskip("torch")
    dims, f, op, _ = setup
    M = 0.2
    prof = ("cosh_4d", 0.3)
    psi = li.random_spinor(dims, 12, 31)
    ev, od = dp.pack_half_spinors(psi, dims)
    Vh = ev.shape[1]

    # FP64: double2 per complex component; FP32 (RHS pairs): float4
    # (re_2q, re_2q+1, im_2q, im_2q+1) per component and pair
    def dev(a):
        if prec == "fp64":
            return torch.from_numpy(np.ascontiguousarray(a).view(np.float64)).cuda()
        pr = a.reshape(12, Vh, 6, 2)
        b = np.stack([pr.real[..., 0], pr.real[..., 1], pr.imag[..., 0], pr.imag[..., 1]], -1)
        return torch.from_numpy(np.ascontiguousarray(b.astype(np.float32))).cuda()

    def host(t):
        if prec == "fp64":
            return t.cpu().numpy().view(np.complex128).reshape(12, Vh, 12)
        b = t.cpu().numpy().reshape(12, Vh, 6, 4).astype(np.float64)
        z = np.stack([b[..., 0] + 1j * b[..., 2], b[..., 1] + 1j * b[..., 3]], -1)
        return z.reshape(12, Vh, 12)

    xin = dev(od)
    outs = []
    for r, stages, block in rpts:
        out = torch.zeros_like(xin)
        dp.dp_dslash_dev(ctx, f, M, prof, prec, c12, 0, xin.data_ptr(), out.data_ptr(), 12,
                         block, r, 1, stages=stages)
        torch.cuda.synchronize()
        outs.append(host(out))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    full_out = dp.unpack_half_spinors(outs[0], np.zeros_like(outs[0]), dims)
    psi_odd = dp.unpack_half_spinors(np.zeros_like(ev), od, dims)
    lhs = (4 + M) * full_out + op.clover(full_out)
    rhs = op.hop(psi_odd, (prof[0], prof[1], (0, 0, 0, 0)))
    t, z, y, x = np.indices(oracle.array_shape(dims))
    even = ((t + x + y + z) % 2) == 0
    assert per_site_rel(lhs[:, even], rhs[:, even]) < 10 * tol


def test_full_size_48x24_fp32_hop(ctx):
    """One multi-RHS FP32 hopping application on the 48x24^3 heavy-quark
    lattice (eps = 0.3, seed 1), all sites compared with the oracle."""
    dims = (48, 24, 24, 24)
    U = li.su3_links(dims, 0.3, 1)
    f = dp.dp_field_load(ctx, U, dims, -1)
    psi = li.random_spinor(dims, 2, 21)
    prof = ("cosh_t", 0.4)
    got = dp.dp_apply(ctx, f, "hop", 0.0, prof, (0, 0, 0, 0), "mixed_fp32", psi, compress12=1)
    op = oracle.WilsonClover(U, dims, 0.0, -1)
    ref = op.hop(psi, ("cosh_t", 0.4, (0, 0, 0, 0)))
    assert per_site_rel(got, ref) < 1e-6
    got64 = dp.dp_apply(ctx, f, "hop", 0.0, prof, (0, 0, 0, 0), "fp64", psi[:1])
    assert per_site_rel(got64, ref[:1]) < 1e-13
    dp.dp_field_free(ctx, f)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed_fp32", 1e-6)])
def test_dirichlet_time_boundary_operator(ctx, prec, tol):
    """bc_t = 0: no quark hop across t = T-1 <-> 0 (Schroedinger-functional-like
    setting), hopping term and full operator with the exp profile."""
    dims = (8, 4, 6, 4)
    U = field(dims, 0.5, 13)
    f = dp.dp_field_load(ctx, U, dims, 0)
    dp.dp_field_set_csw(ctx, f, 1.7)
    op = oracle.WilsonClover(U, dims, 1.7, 0)
    psi = li.random_spinor(dims, 2, 14)
    prof = ("exp_t", 0.4, (0, 1, 2, 3))
    got = dp.dp_apply(ctx, f, "hop", 0.0, prof[:2], prof[2], prec, psi)
    assert per_site_rel(got, op.hop(psi, prof)) < tol
    got = dp.dp_apply(ctx, f, "full", 0.2, prof[:2], prof[2], prec, psi)
    assert per_site_rel(got, op.apply(psi, 0.2, prof)) < tol
    dp.dp_field_free(ctx, f)


def test_tune_set_fixes_the_launch_shape(ctx, setup):
    """A shape set with dp_tune_set is the one the tuned-or-default launch
    uses (bit-identical to the explicit launch); shapes that cannot serve the
    RHS count are refused."""
    torch = pytest.importorskip("torch")
    dims, f, op, _ = setup
    nb = dp.dp_spinor_bytes(ctx, f, "mixed_fp32", 12)
    a = torch.randn(nb // 4, device="cuda")
    explicit, tuned = torch.zeros_like(a), torch.zeros_like(a)
    for shape in [(128, 2, 6), (64, 2, 2), (64, 4, 0)]:
        dp.dp_tune_set(ctx, f, "mixed_fp32", 1, 12, *shape)
        dp.dp_dslash_dev(ctx, f, 0.3, ("cosh_t", 0.4), "mixed_fp32", 1, 0, a.data_ptr(),
                         explicit.data_ptr(), 12, shape[0], shape[1], 1, stages=shape[2])
        dp.dp_dslash_dev(ctx, f, 0.3, ("cosh_t", 0.4), "mixed_fp32", 1, 0, a.data_ptr(),
                         tuned.data_ptr(), 12, 0, 0, 1, stages=-1)
        torch.cuda.synchronize()
        assert torch.equal(explicit, tuned)
    for bad in [(100, 2, 6), (64, 1, 0), (64, 2, 7), (256, 2, 6)]:
        with pytest.raises(dp.DpError):
            dp.dp_tune_set(ctx, f, "mixed_fp32", 1, 12, *bad)
    dp.dp_autotune(ctx, f, "mixed_fp32", 1, 12)


def test_full_size_48x24_schur_launch_in_the_benchmark_shape(ctx):
    """The benchmark's launch at its full size: 48x24^3 heavy-quark lattice
    (eps = 0.3, seed 1, c_sw = 1.7, M = 0.5, cosh alpha0 = 0.4), 12 RHS in
    the spinor-staged kernel with 128 threads (the tuned shape),
    out_e = A_ee^-1 D_eo psi_o, checked through A_ee out_e = D_eo psi_o at
    every even site against the oracle (hop and clover terms), and
    bit-identical to the direct kernel."""
    torch = pytest.importorskip("torch")
    dims = (48, 24, 24, 24)
    U = li.su3_links(dims, 0.3, 1)
    f = dp.dp_field_load(ctx, U, dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    M, prof = 0.5, ("cosh_t", 0.4)
    psi = li.random_spinor(dims, 12, 33)
    ev, od = dp.pack_half_spinors(psi, dims)
    del psi
    Vh = ev.shape[1]
    pr = od.reshape(12, Vh, 6, 2)
    b = np.stack([pr.real[..., 0], pr.real[..., 1], pr.imag[..., 0], pr.imag[..., 1]], -1)
    xin = torch.from_numpy(np.ascontiguousarray(b.astype(np.float32))).cuda()
    del b, pr
    outs = []
    for block, rpt, stages in [(128, 2, 6), (64, 2, 0)]:
        out = torch.zeros_like(xin)
        dp.dp_dslash_dev(ctx, f, M, prof, "mixed_fp32", 1, 0, xin.data_ptr(), out.data_ptr(), 12,
                         block, rpt, 1, stages=stages)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    o = outs[0].reshape(12, Vh, 6, 4).astype(np.float64)
    got = np.stack([o[..., 0] + 1j * o[..., 2], o[..., 1] + 1j * o[..., 3]], -1).reshape(12, Vh, 12)
    del outs, o
    full_out = dp.unpack_half_spinors(got, np.zeros_like(got), dims)
    psi_odd = dp.unpack_half_spinors(np.zeros_like(od), od, dims)
    op = oracle.WilsonClover(U, dims, 1.7, -1)
    lhs = (4 + M) * full_out + op.clover(full_out)
    rhs = op.hop(psi_odd, (prof[0], prof[1], (0, 0, 0, 0)))
    t, z, y, x = np.indices(oracle.array_shape(dims))
    even = ((t + x + y + z) % 2) == 0
    assert per_site_rel(lhs[:, even], rhs[:, even]) < 1e-5
    dp.dp_field_free(ctx, f)


def test_full_size_64x32_light_quark_hop(ctx):
    """The largest workload: the light-quark 64x32^3 lattice (eps = 0.5,
    seed 7) with its cosh-4d profile (alpha0 = 0.2) and an off-origin
    source, 2 RHS: FP32 12-real links against the oracle, and FP16 links
    (the configuration's inner solver) against the oracle on the links as
    the 16-bit storage reproduces them; every site."""
    dims = (64, 32, 32, 32)
    U = li.su3_links(dims, 0.5, 7)
    f = dp.dp_field_load(ctx, U, dims, -1)
    psi = li.random_spinor(dims, 2, 44)
    prof, src = ("cosh_4d", 0.2), (5, 7, 11, 30)
    op = oracle.WilsonClover(U, dims, 0.0, -1)
    ref = op.hop(psi, (prof[0], prof[1], src))
    got = dp.dp_apply(ctx, f, "hop", 0.0, prof, src, "mixed_fp32", psi, compress12=1)
    assert per_site_rel(got, ref) < 1e-6
    del op, ref, got
    op16 = oracle.WilsonClover(oracle.stored_links16(U.reshape(oracle.array_shape(dims) + (4, 3, 3)),
                                                     "fp16"), dims, 0.0, -1)
    got16 = dp.dp_apply(ctx, f, "hop", 0.0, prof, src, "mixed_fp16", psi)
    assert per_site_rel(got16, op16.hop(psi, (prof[0], prof[1], src))) < 1e-6
    dp.dp_field_free(ctx, f)
