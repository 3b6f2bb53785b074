"""Pins of the oracle with a Dirichlet time boundary (bc_t = 0): no quark hop
across t = T-1 <-> 0, the Schroedinger-functional-like setting the paper
recommends the method for (end of Sec. II, profile exp(alpha0 x0)).

Independent checks: removing the seam hop through the boundary factor equals
removing it by zeroing the links that cross the seam (another code path);
gamma5-hermiticity survives; the preconditioned solution restores to the
unpreconditioned one; the free correlator decays over the whole time extent
(no turnover at T/2)."""
import numpy as np

import lattice_inputs as li
import oracle


def test_dirichlet_equals_zeroed_seam_links():
    dims = (6, 4, 4, 4)
    U = li.su3_links(dims, 0.6, 4)
    Uz = U.copy()
    Uz[dims[0] - 1, ..., 0, :, :] = 0  # U_0(t = T-1): the links across the seam
    psi = li.random_spinor(dims, 2, 9)
    for prof in [None, ("exp_t", 0.4, (0, 0, 0, 0)), ("cosh_4d", 0.3, (2, 1, 3, 0))]:
        a = oracle.WilsonClover(U, dims, 0.0, 0).apply(psi, 0.2, prof)
        b = oracle.WilsonClover(Uz, dims, 0.0, 1).apply(psi, 0.2, prof)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
        # and the boundary does change the operator
        c = oracle.WilsonClover(U, dims, 0.0, -1).apply(psi, 0.2, prof)
        assert np.abs(a - c).max() > 1e-3


def test_dirichlet_gamma5_hermiticity():
    dims = (6, 4, 4, 4)
    U = li.su3_links(dims, 0.6, 5)
    op = oracle.WilsonClover(U, dims, 1.7, 0)
    phi = li.random_spinor(dims, 1, 1)
    psi = li.random_spinor(dims, 1, 2)
    g5 = np.diag(oracle.gamma5()).real

    def gam5(v):
        return v * g5[None, None, None, None, None, :, None]

    lhs = np.vdot(phi, op.apply(psi, 0.3))
    rhs = np.conj(np.vdot(psi, gam5(op.apply(gam5(phi), 0.3))))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_dirichlet_restored_equals_unpreconditioned():
    dims = (8, 4, 4, 4)
    U = li.su3_links(dims, 0.4, 6)
    op = oracle.WilsonClover(U, dims, 1.7, 0)
    c0, _, i0 = oracle.solve_point(op, 0.4, "none", 0.0, (0, 1, 2, 3), tol=1e-13)
    c1, _, i1 = oracle.solve_point(op, 0.4, "exp_t", 0.4, (0, 1, 2, 3), tol=1e-13)
    assert i0["converged"] and i1["converged"]
    np.testing.assert_allclose(c1, c0, rtol=1e-9)


def test_free_dirichlet_correlator_decays_over_the_whole_time_extent():
    """Antiperiodic: C_PP(y0) turns over at T/2; Dirichlet: it falls all the
    way to T-1 (source on the first slice)."""
    dims = (12, 4, 4, 4)
    U = li.unit_links(dims)
    cd, _, _ = oracle.solve_point(oracle.WilsonClover(U, dims, 0.0, 0), 0.3, "none", 0.0,
                                  (0, 0, 0, 0), tol=1e-13)
    ca, _, _ = oracle.solve_point(oracle.WilsonClover(U, dims, 0.0, -1), 0.3, "none", 0.0,
                                  (0, 0, 0, 0), tol=1e-13)
    d = -np.asarray(cd)
    a = -np.asarray(ca)
    assert np.all(np.diff(d) < 0)
    assert a[-1] > a[dims[0] // 2]
