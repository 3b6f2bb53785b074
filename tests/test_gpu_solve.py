"""GPU solves (source scaling, Schur solve, restore, contraction) against the
oracle, through the C ABI.

Tolerance: per-time-slice relative deviation of C_PP(y0) <= 1e-6 out to
y0 = T/2, against the oracle's tight-residue (1e-13) solve or, in the free
theory, the exact momentum-space propagator.
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
import paper_1006_4028_gb300 as dp
from gpu_common import field, per_site_rel, require_gpu, slice_rel

pytestmark = pytest.mark.gpu

MIXED = {"prec": "mixed_fp32", "compress12": 1, "batched": 1, "use_graph": 1}
MIXED_NOGRAPH = {"prec": "mixed_fp32", "compress12": 0, "batched": 1, "use_graph": 0}
PLAIN = {"prec": "fp64", "batched": 0, "use_graph": 0}
FP64_BATCHED = {"prec": "fp64", "batched": 1, "use_graph": 1}
# 16-bit links in the inner solver; the FP64 outer loop still fixes the answer
MIXED_FP16 = {"prec": "mixed_fp16", "batched": 1, "use_graph": 1}
MIXED_BF16 = {"prec": "mixed_bf16", "batched": 1, "use_graph": 0}
# CG on the normal equations (the alternative Krylov solver)
CGNE_MIXED = {"prec": "mixed_fp32", "solver": "cgne", "batched": 1, "use_graph": 1}
CGNE_FP64 = {"prec": "fp64", "solver": "cgne", "batched": 1, "use_graph": 0}
# the outer loop's Schur operator in double-float (two FP32 per real)
MIXED_DF = {"prec": "mixed_fp32", "batched": 1, "use_graph": 1, "outer_df": 1}
# the paper's solver: GCR preconditioned by the Schwarz alternating procedure
SAP_GCR = {"prec": "mixed_fp32", "solver": "sap_gcr", "batched": 1, "use_graph": 0}


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    c = dp.dp_create(0)
    yield c
    dp.dp_destroy(c)


@pytest.mark.parametrize("opts", [MIXED, PLAIN, FP64_BATCHED, SAP_GCR])
def test_free_16x8_exp_profile_matches_momentum_space(ctx, opts):
    """Free field 16x8^3, antiperiodic time, M = 0.5, exp(alpha0 y0) with
    alpha0 = 0.4, point source at the origin, r = 1e-11."""
    dims = (16, 8, 8, 8)
    f = dp.dp_field_load(ctx, li.unit_links(dims), dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    cpp, _, info = dp.dp_solve_point(ctx, f, 0.5, ("exp_t", 0.4), (0, 0, 0, 0), 1e-11, opts, T=16)
    exact = oracle.free_cpp(dims, 0.5)
    assert info["status"] == 0
    assert info["true_rel_residue"] < 1e-10
    assert slice_rel(cpp, exact, 8) < 1e-6
    if opts["prec"] == "fp64":
        assert slice_rel(cpp, exact, 15) < 1e-9
    dp.dp_field_free(ctx, f)


@pytest.fixture(scope="module")
def inter(ctx):
    dims = (12, 4, 4, 6)
    U = field(dims, 0.3, 1)
    f = dp.dp_field_load(ctx, U, dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    op = oracle.WilsonClover(U, dims, 1.7, -1)
    return dims, f, op


CASES = [(0.5, ("cosh_t", 0.4), (0, 0, 0, 0)), (0.8, ("cosh_t", 0.5), (3, 1, 2, 0)),
         (0.1, ("cosh_4d", 0.2), (5, 2, 1, 3)), (0.5, ("none", 0.0), (1, 0, 0, 1)),
         (0.5, ("exp_t", 0.3), (2, 3, 3, 5))]


@pytest.mark.parametrize("M,prof,src", CASES)
@pytest.mark.parametrize("opts", [MIXED, MIXED_NOGRAPH, PLAIN, MIXED_FP16, MIXED_BF16, CGNE_MIXED,
                                  CGNE_FP64, MIXED_DF, SAP_GCR])
def test_interacting_solve_matches_oracle(ctx, inter, M, prof, src, opts):
    dims, f, op = inter
    T, V = dims[0], int(np.prod(dims))
    ref, Sref, oinfo = oracle.solve_point(op, M, prof[0], prof[1], src, tol=1e-13)
    assert oinfo["converged"]
    cpp, prop, info = dp.dp_solve_point(ctx, f, M, prof, src, 1e-11, opts, T=T, V=V, want_prop=True)
    assert info["status"] == 0
    assert slice_rel(cpp, ref, T // 2) < 1e-6
    # the restored propagator itself
    got = prop.reshape((12,) + oracle.array_shape(dims) + (4, 3))
    assert per_site_rel(got, Sref) < 1e-5


@pytest.mark.parametrize("r", [1e-10, 1e-12])
def test_double_float_outer_true_residual_fp64(ctx, inter, r):
    """The double-float outer operator decides convergence; the oracle's FP64
    operator then measures the true residual of the returned propagator:
    |eta - (D+M) S| / |eta| <= 1.5 r per source component (no profile, so the
    restored S solves the unpreconditioned system of the same residue)."""
    dims, f, op = inter
    T, V = dims[0], int(np.prod(dims))
    src = (2, 1, 0, 3)
    cpp, prop, info = dp.dp_solve_point(ctx, f, 0.3, ("none", 0.0), src, r, MIXED_DF, T=T, V=V,
                                        want_prop=True)
    assert info["status"] == 0
    S = prop.reshape((12,) + oracle.array_shape(dims) + (4, 3))
    eta = oracle.point_sources(dims, src)
    res = eta - op.apply(S, 0.3)
    rel = np.linalg.norm(res.reshape(12, -1), axis=1) / np.linalg.norm(eta.reshape(12, -1), axis=1)
    assert rel.max() < 1.5 * r
    # and the same solve with the FP64 outer operator agrees per time slice
    cpp64, _, _ = dp.dp_solve_point(ctx, f, 0.3, ("none", 0.0), src, r, MIXED, T=T)
    assert slice_rel(cpp, cpp64, T // 2) < 1e3 * r


@pytest.mark.parametrize("opts", [MIXED, PLAIN])
def test_dirichlet_time_boundary_solve(ctx, opts):
    """Dirichlet time boundary with the exp profile (the Schroedinger-functional
    use the paper recommends), source on the first slice: C_PP over the whole
    time extent against the oracle."""
    dims = (12, 4, 4, 6)
    U = field(dims, 0.3, 8)
    f = dp.dp_field_load(ctx, U, dims, 0)
    dp.dp_field_set_csw(ctx, f, 1.7)
    op = oracle.WilsonClover(U, dims, 1.7, 0)
    src = (0, 1, 2, 3)
    ref, _, oinfo = oracle.solve_point(op, 0.5, "exp_t", 0.4, src, tol=1e-13)
    assert oinfo["converged"]
    cpp, _, info = dp.dp_solve_point(ctx, f, 0.5, ("exp_t", 0.4), src, 1e-11, opts, T=12)
    assert info["status"] == 0
    assert slice_rel(cpp, ref, 11) < 1e-6
    dp.dp_field_free(ctx, f)


@pytest.mark.parametrize("opts", [MIXED, PLAIN])
def test_cap_and_pcac_mass_match_oracle(ctx, inter, opts):
    """C_AP from the same restored propagator as C_PP, against the oracle's
    contraction of its tight solve; the PCAC mass formed from both."""
    dims, f, op = inter
    T = dims[0]
    src = (3, 1, 2, 0)
    ref_cpp, _, oinfo = oracle.solve_point(op, 0.5, "cosh_t", 0.4, src, tol=1e-13)
    ref_cap = oinfo["cap"]
    cpp, cap, info = dp.dp_solve_point_corr(ctx, f, 0.5, ("cosh_t", 0.4), src, 1e-11, opts, T=T)
    assert info["status"] == 0
    assert slice_rel(cpp, ref_cpp, T // 2) < 1e-6
    scale = np.abs(ref_cap[: T // 2 + 1]).max()
    assert np.abs(cap[: T // 2 + 1] - ref_cap[: T // 2 + 1]).max() < 1e-6 * scale
    m_gpu = dp.dp_pcac_mass(cpp, cap)[2: T // 2]
    m_ref = oracle.pcac_mass(ref_cpp, ref_cap)[2: T // 2]
    assert np.abs(m_gpu - m_ref).max() < 1e-5 * np.abs(m_ref).max()


def test_heavy_light_correlator_matches_oracle(ctx, inter):
    """Heavy (cosh profile) and light (cosh-4d profile) quark from one source:
    each C_PP and the complex heavy-light correlator against the oracle."""
    dims, f, op = inter
    T = dims[0]
    src = (3, 1, 2, 0)
    ch, Sh, _ = oracle.solve_point(op, 0.6, "cosh_t", 0.4, src, tol=1e-13)
    cl, Sl, _ = oracle.solve_point(op, 0.1, "cosh_4d", 0.2, src, tol=1e-13)
    ref = oracle.contract_hl(Sh, Sl, dims, src[0])
    cpp, hl, infos = dp.dp_solve_point_hl(ctx, f, 0.6, ("cosh_t", 0.4), 0.1, ("cosh_4d", 0.2), src,
                                          1e-12, MIXED, T=T)
    assert all(i["status"] == 0 for i in infos)
    assert slice_rel(cpp[0], ch, T // 2) < 1e-6 and slice_rel(cpp[1], cl, T // 2) < 1e-6
    scale = np.abs(ref[: T // 2 + 1]).max()
    assert np.abs(hl[: T // 2 + 1] - ref[: T // 2 + 1]).max() < 1e-6 * scale
    # equal masses and profiles: the heavy-light correlator is C_PP
    cpp2, hl2, _ = dp.dp_solve_point_hl(ctx, f, 0.6, ("cosh_t", 0.4), 0.6, ("cosh_t", 0.4), src,
                                        1e-12, MIXED, T=T)
    assert np.abs(hl2 - cpp2[0]).max() < 1e-12 * np.abs(cpp2[0]).max()


def test_multi_mass_batch_equals_single_solves(ctx, inter):
    dims, f, op = inter
    T = dims[0]
    Ms = [0.1, 0.5, 0.8]
    profs = [("cosh_4d", 0.2), ("cosh_t", 0.4), ("cosh_t", 0.5)]
    src = (2, 1, 0, 3)
    multi, _, infos = dp.dp_solve_point_multi(ctx, f, Ms, profs, src, 1e-11, MIXED, T=T)
    for k in range(3):
        single, _, _ = dp.dp_solve_point(ctx, f, Ms[k], profs[k], src, 1e-11, MIXED, T=T)
        assert slice_rel(multi[k], single, T // 2) < 1e-8
        ref, _, _ = oracle.solve_point(op, Ms[k], profs[k][0], profs[k][1], src, tol=1e-13)
        assert slice_rel(multi[k], ref, T // 2) < 1e-6
        assert infos[k]["status"] == 0


def test_restored_independent_of_profile(ctx, inter):
    """Exact similarity transform: every profile restores the same C_PP."""
    dims, f, op = inter
    T = dims[0]
    base, _, _ = dp.dp_solve_point(ctx, f, 0.5, ("none", 0.0), (0, 0, 0, 0), 1e-12, MIXED, T=T)
    for prof in [("cosh_t", 0.3), ("cosh_t", 0.5), ("exp_t", 0.4), ("cosh_4d", 0.2)]:
        c, _, _ = dp.dp_solve_point(ctx, f, 0.5, prof, (0, 0, 0, 0), 1e-12, MIXED, T=T)
        assert slice_rel(c, base, T // 2) < 1e-7


def test_loose_residue_heavy_quark_effect(ctx):
    """Sec. II: at r = 1e-6 the unpreconditioned far slices drift; with the
    cosh profile (alpha0 = 0.4) the restored correlator stays accurate.  The
    paper's global stopping rule alone (the library's per-slice check off)
    shows the effect; with the check on (the default) the unpreconditioned
    solve is refined until its far slices hold too."""
    dims = (48, 4, 4, 4)
    f = dp.dp_field_load(ctx, li.unit_links(dims), dims, -1)
    dp.dp_field_set_csw(ctx, f, 0.0)
    exact = oracle.free_cpp(dims, 0.5)
    paper = dict(PLAIN, slice_tol=-1.0)
    loose, _, _ = dp.dp_solve_point(ctx, f, 0.5, ("none", 0.0), (0, 0, 0, 0), 1e-6, paper, T=48)
    prec, _, _ = dp.dp_solve_point(ctx, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-6, paper, T=48)
    e_loose = np.abs(loose / exact - 1)[:25]
    e_prec = np.abs(prec / exact - 1)[:25]
    assert e_loose.max() > 1e-2
    assert e_prec.max() < 1e-4
    checked, _, info = dp.dp_solve_point(ctx, f, 0.5, ("none", 0.0), (0, 0, 0, 0), 1e-6, PLAIN,
                                         T=48)
    assert info["status"] == 0 and info["slice_residue"] <= 1e-5
    assert np.abs(checked / exact - 1)[:25].max() < 1e-4
    dp.dp_field_free(ctx, f)


def test_not_converged_and_bad_arguments(ctx, inter):
    dims, f, op = inter
    T = dims[0]
    o = dict(MIXED, max_iter=3)
    with pytest.raises(dp.DpError) as e:
        dp.dp_solve_point(ctx, f, 0.05, ("none", 0.0), (0, 0, 0, 0), 1e-12, o, T=T, allow=())
    assert e.value.status == 3
    cpp, _, info = dp.dp_solve_point(ctx, f, 0.05, ("none", 0.0), (0, 0, 0, 0), 1e-12, o, T=T)
    assert info["status"] == 3 and info["iters_inner"] <= 3 * 40
    for bad in [dict(src=(12, 0, 0, 0)), dict(r=0.0), dict(r=1.5), dict(M=float("nan"))]:
        args = dict(M=0.5, src=(0, 0, 0, 0), r=1e-8)
        args.update(bad)
        with pytest.raises(dp.DpError) as e:
            dp.dp_solve_point(ctx, f, args["M"], ("none", 0.0), args["src"], args["r"], MIXED, T=T)
        assert e.value.status == 1
    for bad_opts in [dict(MIXED, prec=7), dict(MIXED, solver=5), dict(MIXED, inner_tol=1.5)]:
        with pytest.raises(dp.DpError) as e:
            dp.dp_solve_point(ctx, f, 0.5, ("none", 0.0), (0, 0, 0, 0), 1e-8, bad_opts, T=T)
        assert e.value.status == 1


def test_device_output_and_timing(ctx, inter):
    torch = pytest.importorskip("torch")
    dims, f, op = inter
    T = dims[0]
    out = torch.zeros(2 * T, dtype=torch.float64, device="cuda")
    dp.dp_timing_enable(ctx, True)
    dp.dp_timing_reset(ctx)
    n0 = dp.dp_launch_count(ctx)
    infos = dp.dp_solve_point_dev(ctx, f, [0.5, 0.8], [("cosh_t", 0.4), ("cosh_t", 0.5)],
                                  (0, 0, 0, 0), 1e-10, out.data_ptr(), MIXED)
    torch.cuda.synchronize()
    launches, ms = dp.dp_timing_get(ctx, "dslash_fp32")
    dp.dp_timing_enable(ctx, False)
    assert launches > 0 and ms > 0
    assert dp.dp_launch_count(ctx) - n0 > launches
    host, _, _ = dp.dp_solve_point_multi(ctx, f, [0.5, 0.8], [("cosh_t", 0.4), ("cosh_t", 0.5)],
                                         (0, 0, 0, 0), 1e-10, MIXED, T=T)
    np.testing.assert_array_equal(out.cpu().numpy().reshape(2, T), host)
    assert all(i["status"] == 0 for i in infos)


def test_pool_keeps_memory_and_trim(ctx, inter):
    """The context's pool reuses a solve's freed work vectors; results do not
    depend on whether the memory was trimmed in between (deterministic)."""
    dims, f, op = inter
    held = dp.dp_device_bytes(ctx)
    a, _, ia = dp.dp_solve_point(ctx, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-10, MIXED, T=dims[0])
    assert dp.dp_device_bytes(ctx) <= held + (1 << 30)  # work vectors returned after the call
    dp.dp_trim(ctx)
    b, _, ib = dp.dp_solve_point(ctx, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-10, MIXED, T=dims[0])
    c, _, _ = dp.dp_solve_point(ctx, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-10, MIXED, T=dims[0])
    assert ia["status"] == 0 and ib["status"] == 0
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(b, c)


def test_effective_mass_fit_of_solved_free_correlator(ctx):
    """C_PP from the GPU solve, analysed by the library's host functions,
    against the oracle's analysis of the exact free correlator."""
    dims = (16, 8, 8, 8)
    f = dp.dp_field_load(ctx, li.unit_links(dims), dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    cpp, _, info = dp.dp_solve_point(ctx, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-11, MIXED, T=16)
    exact = oracle.free_cpp(dims, 0.5)
    assert info["status"] == 0
    got = dp.dp_effective_mass(cpp, "cosh")
    ref = oracle.effective_mass_cosh(exact)
    np.testing.assert_allclose(got[:8], ref[:8], rtol=0, atol=1e-5)
    m, _, _ = dp.dp_fit_correlator(cpp, "cosh", 4, 12)
    mo, _, _ = oracle.fit_correlator(exact, "cosh", 4, 12)
    assert abs(m - mo) < 1e-6
    dp.dp_field_free(ctx, f)


@pytest.mark.parametrize("opts", [MIXED, CGNE_MIXED, SAP_GCR])
@pytest.mark.parametrize("shape", [(128, 2, 6), (96, 2, 6)])
def test_solvers_on_the_spinor_staged_kernel(ctx, opts, shape):
    """BiCGStab, CGNE (whose adjoint's x - g5 D launch also runs on it) and
    SAP+GCR with the tuned shape forced to the spinor-staged kernel, on a
    6x4x6x6 lattice whose 2592 pair-threads leave a ragged last block:
    C_PP against the oracle."""
    dims = (6, 4, 6, 6)
    U = field(dims, 0.3, 5)
    f = dp.dp_field_load(ctx, U, dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    op = oracle.WilsonClover(U, dims, 1.7, -1)
    src = (1, 0, 2, 3)
    ref, _, _ = oracle.solve_point(op, 0.5, "cosh_t", 0.4, src, tol=1e-13)
    dp.dp_tune_set(ctx, f, "mixed_fp32", 1, 12, *shape)
    cpp, _, info = dp.dp_solve_point(ctx, f, 0.5, ("cosh_t", 0.4), src, 1e-10, opts, T=6)
    assert info["status"] == 0 and info["true_rel_residue"] < 1e-10
    assert slice_rel(cpp, ref, 3) < 1e-6
    dp.dp_field_free(ctx, f)


def test_full_size_48x24_solve_matches_stored_oracle(ctx):
    """The benchmark's solve at its full size: 48x24^3 heavy-quark workload,
    point source at the origin, r = 1e-11, FP32 inner BiCGStab on the
    spinor-staged kernel (the tuned shape) in the FP64 outer loop; C_PP per
    time slice out to T/2 against the oracle's stored r = 1e-13 result
    (tests/golden/cpp_48x24_M0.5_cosh0.4.json, written by make_golden.py)."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "cpp_48x24_M0.5_cosh0.4.json")))
    dims = tuple(g["dims"])
    f = dp.dp_field_load(ctx, li.su3_links(dims, g["eps"], g["seed"]), dims, g["bc_t"])
    dp.dp_field_set_csw(ctx, f, g["csw"])
    dp.dp_tune_set(ctx, f, "mixed_fp32", 1, 12, 128, 2, 6)
    cpp, _, info = dp.dp_solve_point(ctx, f, g["M"], (g["profile"], g["alpha0"]), tuple(g["src"]),
                                     1e-11, MIXED, T=dims[0])
    assert info["status"] == 0 and info["true_rel_residue"] < 1e-11
    assert slice_rel(cpp, g["cpp"], dims[0] // 2) < 1e-6
    dp.dp_field_free(ctx, f)


@pytest.mark.parametrize("M,prof", [(0.5, ("cosh_t", 0.4)), (0.1, ("cosh_4d", 0.2)),
                                    (0.5, ("none", 0.0))])
def test_fp32_bicgstab_iterations_track_fp64(ctx, M, prof):
    """The FP32 inner BiCGStab in shadow form (rhat' = Mhat^dag rhat once per
    inner solve; <t, s> and |t|^2 summed in the x - A^-1 D epilogue) makes
    the iterates of the FP64 BiCGStab in exact arithmetic, so at a residue
    one inner solve reaches long before FP32 rounding matters (r = 1e-4)
    their iteration counts agree.  A wrong inner product would cost
    iterations, not accuracy (the FP64 outer loop corrects the answer), so
    the parity tests alone would not see it."""
    dims = (16, 8, 8, 8)
    f = dp.dp_field_load(ctx, field(dims, 0.3, 2), dims, -1)
    dp.dp_field_set_csw(ctx, f, 1.7)
    its = {}
    for prec in ("mixed_fp32", "fp64"):
        o = {"prec": prec, "batched": 1, "use_graph": 0, "slice_tol": -1.0}
        _, _, info = dp.dp_solve_point(ctx, f, M, prof, (0, 0, 0, 0), 1e-4, o, T=dims[0])
        assert info["status"] == 0 and info["iters_outer"] == 1, (prec, info)
        its[prec] = info["iters_inner"]
    assert abs(its["mixed_fp32"] - its["fp64"]) <= 1, its
    dp.dp_field_free(ctx, f)
