"""Pins of the oracle's axial-pseudoscalar correlator C_AP and the PCAC mass
(the paper labels its quark masses by am_PCAC, Sec. II).

Independent checks: time reflection makes the free C_AP odd about the source
(C_AP(T - y0) = -C_AP(y0), zero at y0 = 0 and T/2) while C_PP is even; at
tree level the PCAC mass tends to the bare mass M in the chiral limit (slope
1, the Wilson term vanishes at zero momentum); gauge invariance; and the
restored C_AP does not depend on the preconditioning profile."""
import numpy as np

import lattice_inputs as li
import oracle
from test_oracle_symmetry import gauge_transform


def test_free_cap_is_odd_under_time_reflection():
    dims = (12, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, 0.0, -1)
    cpp, _, info = oracle.solve_point(op, 0.3, "none", 0.0, (0, 0, 0, 0), tol=1e-13)
    cap = info["cap"]
    T = dims[0]
    refl = np.array([cap[(T - t) % T] for t in range(T)])
    assert np.abs(cap + refl).max() < 1e-12 * np.abs(cap).max()
    assert abs(cap[0]) < 1e-12 * np.abs(cap).max() and abs(cap[T // 2]) < 1e-12 * np.abs(cap).max()
    cpp_refl = np.array([cpp[(T - t) % T] for t in range(T)])
    assert np.abs(cpp - cpp_refl).max() < 1e-12 * np.abs(cpp).max()
    assert np.abs(cap).max() > 1e-3 * np.abs(cpp).max()


def test_free_pcac_mass_tends_to_bare_mass():
    """Plateau of m_PCAC(y0) in the free theory: flat, and m/M -> 1 as M -> 0."""
    dims = (20, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, 0.0, -1)
    ratios = []
    for M in (0.01, 0.04):
        cpp, _, info = oracle.solve_point(op, M, "none", 0.0, (0, 0, 0, 0), tol=1e-13)
        m = oracle.pcac_mass(cpp, info["cap"])
        plateau = m[7:10]
        assert np.ptp(plateau) < 5e-3 * abs(plateau.mean())
        ratios.append(plateau.mean() / M)
    assert abs(ratios[0] - 1) < 0.01 and abs(ratios[1] - 1) < 0.04
    assert abs(ratios[0] - 1) < abs(ratios[1] - 1)


def test_cap_gauge_invariant_and_profile_independent():
    dims = (8, 4, 4, 4)
    U = li.su3_links(dims, 0.4, seed=3)
    G = li.random_gauge_transform(dims, seed=4)
    src = (2, 1, 0, 3)
    op = oracle.WilsonClover(U, dims, 1.7)
    _, _, a = oracle.solve_point(op, 0.4, "none", 0.0, src)
    _, _, b = oracle.solve_point(oracle.WilsonClover(gauge_transform(U, G), dims, 1.7), 0.4,
                                 "none", 0.0, src)
    _, _, c = oracle.solve_point(op, 0.4, "cosh_t", 0.4, src)
    scale = np.abs(a["cap"]).max()
    assert np.abs(b["cap"] - a["cap"]).max() < 1e-10 * scale
    assert np.abs(c["cap"] - a["cap"]).max() < 1e-10 * scale


def test_heavy_light_reduces_to_cpp_and_is_gauge_invariant():
    """Equal masses: the heavy-light correlator is C_PP (real); unequal
    masses: gauge invariant, independent of each quark's profile."""
    dims = (8, 4, 4, 4)
    U = li.su3_links(dims, 0.4, seed=3)
    G = li.random_gauge_transform(dims, seed=4)
    src = (2, 1, 0, 3)
    op = oracle.WilsonClover(U, dims, 1.7)
    opg = oracle.WilsonClover(gauge_transform(U, G), dims, 1.7)
    cpp, Sh, _ = oracle.solve_point(op, 0.5, "cosh_t", 0.4, src)
    same = oracle.contract_hl(Sh, Sh, dims, src[0])
    assert np.abs(same - cpp).max() < 1e-13 * np.abs(cpp).max()
    _, Sl, _ = oracle.solve_point(op, 0.1, "none", 0.0, src)
    _, Sl2, _ = oracle.solve_point(op, 0.1, "cosh_4d", 0.2, src)
    _, Shg, _ = oracle.solve_point(opg, 0.5, "cosh_t", 0.4, src)
    _, Slg, _ = oracle.solve_point(opg, 0.1, "none", 0.0, src)
    hl = oracle.contract_hl(Sh, Sl, dims, src[0])
    scale = np.abs(hl).max()
    assert np.abs(oracle.contract_hl(Sh, Sl2, dims, src[0]) - hl).max() < 1e-10 * scale
    assert np.abs(oracle.contract_hl(Shg, Slg, dims, src[0]) - hl).max() < 1e-10 * scale
    # a genuinely different correlator from either C_PP
    cl, _, _ = oracle.solve_point(op, 0.1, "none", 0.0, src)
    assert np.abs(hl.real - cpp).max() > 1e-3 * scale and np.abs(hl.real - cl).max() > 1e-3 * scale
