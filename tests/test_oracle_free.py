"""Free-theory pins of the oracle (U = 1).

* plane waves are eigenvectors of D with the closed-form D(p);
* the solved point-source C_PP equals the exact momentum-space propagator's
  C_PP, with and without the preconditioning profiles (the transform is
  exact, Sec. II "does not introduce any approximation");
* the effective mass sits near the free two-quark energy 2 ln(1+M).
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle


def _plane_wave(dims, n, chi, bc_t):
    T, Lx, Ly, Lz = dims
    t, x, y, z = oracle.site_coords(dims)
    shift0 = 0.5 if bc_t < 0 else 0.0
    p = [2 * np.pi * (n[0] + shift0) / T, 2 * np.pi * n[1] / Lx,
         2 * np.pi * n[2] / Ly, 2 * np.pi * n[3] / Lz]
    phase = np.exp(1j * (p[0] * t + p[1] * x + p[2] * y + p[3] * z))
    return p, phase[..., None, None] * chi[None, None, None, None]


@pytest.mark.parametrize("bc_t", [-1, 1])
def test_plane_wave_eigen_relation(bc_t):
    dims = (6, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=1.9, bc_t=bc_t)
    rng = np.random.default_rng(11)
    M = 0.37
    for n in [(0, 0, 0, 0), (1, 2, 3, 1), (5, 1, 0, 3), (2, 3, 1, 2)]:
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        p, psi = _plane_wave(dims, n, chi, bc_t)
        got = op.apply(psi[None], M)[0]
        Dp = oracle.free_momentum_operator(p, M)
        want = np.einsum("st,...tc->...sc", Dp, psi)
        assert np.abs(got - want).max() < 1e-14 * np.abs(want).max() * 10


@pytest.mark.parametrize(
    "kind,alpha0,src",
    [("none", 0.0, (0, 0, 0, 0)), ("exp_t", 0.4, (0, 0, 0, 0)),
     ("cosh_t", 0.4, (3, 1, 2, 0)), ("cosh_4d", 0.2, (5, 3, 0, 1))],
)
def test_free_cpp_matches_momentum_space(kind, alpha0, src):
    dims = (8, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=1.7, bc_t=-1)
    cpp, _, info = oracle.solve_point(op, 0.5, kind, alpha0, src, tol=1e-14)
    assert info["converged"]
    exact = oracle.free_cpp(dims, 0.5, bc_t=-1)
    assert np.all(cpp < 0)
    assert np.abs(cpp / exact - 1).max() < 1e-12


@pytest.mark.slow
def test_free_cpp_16x8_exp_profile():
    """The free workload 16x8^3, M = 0.5, exp(alpha0 y0) profile, alpha0 = 0.4."""
    dims = (16, 8, 8, 8)
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=1.7, bc_t=-1)
    cpp, _, info = oracle.solve_point(op, 0.5, "exp_t", 0.4, (0, 0, 0, 0), tol=1e-13)
    assert info["converged"]
    exact = oracle.free_cpp(dims, 0.5, bc_t=-1)
    assert np.abs(cpp / exact - 1).max() < 1e-11


@pytest.mark.parametrize("M", [0.5, 0.8])
def test_free_cpp_decay_rate_is_two_quark_pole(M):
    """Far from the source and the boundary the free pseudoscalar correlator
    decays with twice the zero-momentum Wilson quark energy, e^E = 1 + M (r = 1),
    so the effective mass tends to 2 ln(1 + M)."""
    dims = (96, 4, 4, 4)
    meff = oracle.effective_mass(oracle.free_cpp(dims, M))
    assert abs(meff[24] - 2 * np.log(1 + M)) < 1e-5


def test_free_propagator_solves_point_source():
    """The momentum-space S is a Green function: (D+M) S = delta (direct check)."""
    dims = (6, 4, 4, 2)
    M = 0.5
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=0.0, bc_t=-1)
    S = oracle.free_propagator(dims, M)  # (T, Lz, Ly, Lx, 4, 4)
    for sp in range(4):
        psi = np.zeros(oracle.array_shape(dims) + (4, 3), complex)
        psi[..., :, 0] = S[..., :, sp]
        out = op.apply(psi[None], M)[0]
        want = np.zeros_like(out)
        want[0, 0, 0, 0, sp, 0] = 1
        assert np.abs(out - want).max() < 1e-14


def test_stored_free_golden_is_the_oracles():
    """tests/golden/free_16x8_M0.5.json (read by the benchmark's free-theory
    check) holds exactly the oracle's momentum-space C_PP."""
    import json
    import os

    p = os.path.join(os.path.dirname(__file__), "golden", "free_16x8_M0.5.json")
    d = json.load(open(p))
    np.testing.assert_allclose(d["cpp"], oracle.free_cpp(tuple(d["dims"]), d["M"], d["bc_t"]),
                               rtol=1e-14, atol=0)
