"""Pins of the oracle's effective masses and correlator fit.

The paper plots effective masses without writing a definition out; the
oracle takes the log ratio ln[C(y0)/C(y0+1)] and the cosh form for two-sided
decay round a periodic time direction.  Independent checks: exact one- and
two-sided exponentials return their mass at every y0, and in the free theory
the zero-momentum pseudoscalar decays with twice the Wilson quark pole
energy ln(1+M) (r = 1), the value the cosh effective mass reaches once the
non-zero spatial momenta have died out."""
import numpy as np

import oracle


def test_exact_exponentials():
    t = np.arange(24, dtype=float)
    one = -0.3 * np.exp(-0.7 * t)
    np.testing.assert_allclose(oracle.effective_mass(one), 0.7, rtol=0, atol=1e-13)
    two = 2.0 * np.cosh(0.45 * (t - 12))
    m = oracle.effective_mass_cosh(two)
    np.testing.assert_allclose(m[np.isfinite(m)], 0.45, rtol=0, atol=1e-12)
    assert np.isfinite(m).sum() == 23
    mf, A, rms = oracle.fit_correlator(one, "exp", 3, 15)
    assert abs(mf - 0.7) < 1e-12 and abs(A + 0.3) < 1e-12 and rms < 1e-13
    mf, A, rms = oracle.fit_correlator(two, "cosh", 4, 20)
    assert abs(mf - 0.45) < 1e-12 and abs(A / np.exp(0.45 * 12) - 1) < 1e-11 and rms < 1e-13


def test_free_pseudoscalar_decays_with_twice_the_pole_energy():
    dims = (64, 4, 4, 4)
    M = 0.5
    c = oracle.free_cpp(dims, M)
    E2 = 2 * np.log(1 + M)
    mc = oracle.effective_mass_cosh(c)
    assert np.abs(mc[20:40] - E2).max() < 5e-11
    ml = oracle.effective_mass(c)
    assert np.abs(ml[15:22] - E2).max() < 1e-6
    # the log ratio turns over at T/2, the cosh form does not
    assert ml[40] < 0 and abs(mc[40] - E2) < 5e-11
    m, _, rms = oracle.fit_correlator(c, "cosh", 20, 44)
    assert abs(m - E2) < 1e-10 and rms < 1e-9
    # excited (non-zero momentum) states pull the early window up
    assert mc[4] > E2 + 1e-4


def test_undefined_ratios_are_nan():
    c = np.array([-1.0, -0.5, 0.2, 0.1, -0.05])
    m = oracle.effective_mass_cosh(c)
    assert np.isfinite(m[0]) and np.isnan(m[1]) and np.isnan(m[3])
