"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
the header declares, and its host-side profile/hop tables agree with the
oracle's independent implementation.  No GPU compute is called here."""
import re

import numpy as np
import pytest

import lattice_inputs as li
import oracle
import paper_1006_4028_gb300 as dp
from paper_1006_4028_gb300 import build as dpbuild


@pytest.fixture(scope="module")
def lib():
    dpbuild.build()
    return dp.load()


def declared_functions():
    src = open(dpbuild.INCLUDE + "/dpre.h").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(dp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["dp_create", "dp_destroy", "dp_last_error", "dp_field_load", "dp_field_set_csw",
                 "dp_field_free", "dp_solve_point", "dp_submit", "dp_wait"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


KINDS = [("none", 0.0), ("exp_t", 0.4), ("cosh_t", 0.3), ("cosh_4d", 0.2)]


@pytest.mark.parametrize("kind,alpha0", KINDS)
@pytest.mark.parametrize("src", [(0, 0, 0, 0), (5, 3, 1, 2)])
@pytest.mark.parametrize("bc_t", [-1, 1, 0])
def test_host_profile_tables_match_oracle(lib, kind, alpha0, src, bc_t):
    dims = (16, 8, 4, 6)
    alpha, hop = dp.dp_profile_tables(dims, bc_t, (kind, alpha0), src)
    ref_al = oracle.profile_alpha(kind, alpha0, dims, src)
    fwd, bwd, _ = oracle.hop_tables(ref_al, dims, bc_t)
    for mu in range(4):
        L = dims[mu]
        np.testing.assert_allclose(alpha[mu, :L], ref_al[mu], rtol=1e-15, atol=0)
        np.testing.assert_allclose(hop[mu, 0, :L], -0.5 * fwd[mu, :L], rtol=1e-14, atol=0)
        np.testing.assert_allclose(hop[mu, 1, :L], -0.5 * bwd[mu, :L], rtol=1e-14, atol=0)


def test_host_profile_table_kind(lib):
    dims = (8, 4, 4, 4)
    rng = np.random.default_rng(1)
    tabs = [rng.uniform(0.5, 2.0, size=d) for d in dims]
    alpha, hop = dp.dp_profile_tables(dims, -1, ("table", 0.0, tabs))
    fwd, bwd, _ = oracle.hop_tables(tabs, dims, -1)
    for mu in range(4):
        np.testing.assert_allclose(alpha[mu, :dims[mu]], tabs[mu], rtol=0)
        np.testing.assert_allclose(hop[mu, 0, :dims[mu]], -0.5 * fwd[mu, :dims[mu]], rtol=1e-15)


@pytest.mark.parametrize("dims", [(7, 4, 4, 4), (8, 3, 4, 4), (8, 4, 4, 1), (300, 4, 4, 4)])
def test_host_rejects_bad_geometry(lib, dims):
    with pytest.raises(dp.DpError) as e:
        dp.dp_profile_tables(dims, -1, ("none", 0.0))
    assert e.value.status == 1


def test_host_rejects_bad_profiles(lib):
    with pytest.raises(dp.DpError):
        dp.dp_profile_tables((8, 4, 4, 4), -1, ("exp_t", float("nan")))
    with pytest.raises(dp.DpError):
        dp.dp_profile_tables((8, 4, 4, 4), -1, ("table", 0.0, [np.zeros(8)] + [np.ones(4)] * 3))
    with pytest.raises(dp.DpError):
        dp.dp_profile_tables((8, 4, 4, 4), 2, ("none", 0.0))
    with pytest.raises(dp.DpError):
        dp.dp_profile_tables((8, 4, 4, 4), -1, ("none", 0.0), (8, 0, 0, 0))


def test_pack_half_spinors_layout():
    """Host marshalling into the packed even/odd layout [12][V/2][n]."""
    import lattice_inputs as li

    dims = (4, 2, 4, 2)
    S = li.random_spinor(dims, 3, 1)
    ev, od = dp.pack_half_spinors(S, dims)
    T, Lx, Ly, Lz = dims
    seen = 0
    for t in range(T):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    i = ((t * Lz + z) * Ly + y) * Lx + x
                    half = ev if (t + x + y + z) % 2 == 0 else od
                    np.testing.assert_array_equal(half[:, i >> 1, :],
                                                  S[:, t, z, y, x].reshape(3, 12).T)
                    seen += 1
    assert seen == 64 and ev.shape == (12, 32, 3)


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dp.DpError) as e:
        dp.dp_create(0)
    assert e.value.status == 8
    assert "device" in e.value.message


@pytest.mark.parametrize("kind,alpha0", KINDS)
@pytest.mark.parametrize("bc_t", [-1, 1])
def test_reciprocal_profile_hop_factors(lib, kind, alpha0, bc_t):
    """The adjoint operator's hopping part uses the reciprocal profile
    1/alpha_B; the solver forms its hop factors as (1/4) / (the profile's own),
    which must equal the oracle's factors for the profile 1/alpha_B."""
    dims = (12, 6, 4, 8)
    src = (3, 1, 2, 5)
    _, hop = dp.dp_profile_tables(dims, bc_t, (kind, alpha0), src)
    ref_al = oracle.profile_alpha(kind, alpha0, dims, src)
    fwd, bwd, _ = oracle.hop_tables([1.0 / a for a in ref_al], dims, bc_t)
    for mu in range(4):
        L = dims[mu]
        np.testing.assert_allclose(0.25 / hop[mu, 0, :L], -0.5 * fwd[mu, :L], rtol=1e-14, atol=0)
        np.testing.assert_allclose(0.25 / hop[mu, 1, :L], -0.5 * bwd[mu, :L], rtol=1e-14, atol=0)


def test_effective_mass_and_fit_match_oracle(lib):
    """Host-side correlator analysis of the library (bisection, scan and
    golden-section search) against the oracle's (Brent, Levenberg-Marquardt)
    on the free 64x4^3 correlator and on exact exponentials."""
    c = oracle.free_cpp((64, 4, 4, 4), 0.5)
    for kind, ref in (("log", oracle.effective_mass(c)), ("cosh", oracle.effective_mass_cosh(c))):
        got = dp.dp_effective_mass(c, kind)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        ok = np.isfinite(ref)
        np.testing.assert_allclose(got[ok], ref[ok], rtol=1e-12, atol=1e-13)
    for kind, t0, t1 in (("cosh", 20, 44), ("cosh", 6, 30), ("exp", 10, 20)):
        m, A, rms = dp.dp_fit_correlator(c, kind, t0, t1)
        mo, Ao, rmso = oracle.fit_correlator(c, kind, t0, t1)
        assert abs(m - mo) < 1e-9 * mo and abs(A - Ao) < 1e-8 * abs(Ao)
        assert abs(rms - rmso) < 1e-9 + 1e-6 * rmso
    t = np.arange(24, dtype=float)
    m, A, rms = dp.dp_fit_correlator(2.0 * np.cosh(0.45 * (t - 12)), "cosh", 3, 21)
    assert abs(m - 0.45) < 1e-12 and rms < 1e-13


def test_analysis_rejects_bad_windows(lib):
    c = np.array([-1.0, -0.5, 0.2, 0.1, -0.05])
    with pytest.raises(dp.DpError):
        dp.dp_fit_correlator(c, "exp", 0, 3)      # sign change
    with pytest.raises(dp.DpError):
        dp.dp_fit_correlator(c, "exp", 3, 3)      # one point
    with pytest.raises(dp.DpError):
        dp.dp_fit_correlator(c, "cosh", 2, 5)     # past T
    m = dp.dp_effective_mass(c, "cosh")
    assert np.isfinite(m[0]) and np.isnan(m[1])


def test_pcac_mass_matches_oracle(lib):
    """The library's PCAC ratio (host function) against the oracle's on the
    free correlators (whose plateau the oracle pins to the bare mass), and its
    NaN ends and argument checks."""
    dims, M = (16, 4, 4, 4), 0.05
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=1.7, bc_t=-1)
    cpp, _, info = oracle.solve_point(op, M, "none", 0.0, (0, 0, 0, 0), tol=1e-13)
    got = dp.dp_pcac_mass(cpp, info["cap"])
    ref = oracle.pcac_mass(cpp, info["cap"])
    assert np.isnan(got[0]) and np.isnan(got[-1])
    np.testing.assert_allclose(got[1:-1], ref[1:-1], rtol=1e-13, atol=0)
    with pytest.raises(dp.DpError):
        dp.dp_pcac_mass(cpp[:2], info["cap"][:2])
