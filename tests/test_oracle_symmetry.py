"""Symmetry pins of the oracle operator on interacting synthetic fields.

* gamma_5-hermiticity  <phi, D psi> = <gamma5 D gamma5 phi, psi>;
* with the profile:    D'(alpha_B)^dag = gamma5 D'(1/alpha_B) gamma5;
* gauge covariance     D[U^G] G psi = G D[U] psi (Haar-random G);
* the preconditioned operator is the similarity transform A (D+M) A^-1 with
  A = diag(alpha_B) (Sec. II eqs. redeft/linsysprec, Sec. III eq. redefa),
  checked as dense matrices, and its forward-hop coefficient is
  alpha_B(x_mu)/alpha_B(x_mu+1) (the modified derivative of Sec. II in the
  alpha_B = 1/alpha orientation).
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from test_oracle_clover import gauge_transform

G5 = np.diag([1.0, 1.0, -1.0, -1.0])


def g5(psi):
    return np.einsum("st,...tc->...sc", G5, psi)


@pytest.mark.parametrize("csw,bc_t", [(0.0, -1), (1.7, -1), (1.9, 1)])
def test_gamma5_hermiticity(csw, bc_t):
    dims = (4, 4, 4, 6)
    op = oracle.WilsonClover(li.su3_links(dims, 0.5, seed=7), dims, csw, bc_t)
    phi = li.random_spinor(dims, 1, 21)
    psi = li.random_spinor(dims, 1, 22)
    M = 0.1
    lhs = np.vdot(phi, op.apply(psi, M))
    rhs = np.vdot(g5(op.apply(g5(phi), M)), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("kind,alpha0", [("cosh_t", 0.4), ("exp_t", 0.3), ("cosh_4d", 0.2)])
def test_preconditioned_adjoint_uses_reciprocal_profile(kind, alpha0):
    dims = (6, 4, 4, 4)
    op = oracle.WilsonClover(li.su3_links(dims, 0.3, seed=8), dims, 1.7, -1)
    src = (2, 1, 3, 0)
    al = oracle.profile_alpha(kind, alpha0, dims, src)
    inv = [1.0 / a for a in al]
    phi = li.random_spinor(dims, 1, 31)
    psi = li.random_spinor(dims, 1, 32)
    M = 0.5
    lhs = np.vdot(phi, op.apply(psi, M, ("table", 0, src, al)))
    rhs = np.vdot(g5(op.apply(g5(phi), M, ("table", 0, src, inv))), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_gauge_covariance():
    dims = (4, 6, 4, 4)
    U = li.su3_links(dims, 0.5, seed=12)
    G = li.random_gauge_transform(dims, seed=13)
    psi = li.random_spinor(dims, 1, 14)[0]
    M = 0.2
    prof = ("cosh_4d", 0.3, (1, 2, 0, 3))
    op = oracle.WilsonClover(U, dims, 1.7, -1)
    opG = oracle.WilsonClover(gauge_transform(U, G), dims, 1.7, -1)
    Gpsi = np.einsum("...ab,...sb->...sa", G, psi)
    lhs = opG.apply(Gpsi[None], M, prof)[0]
    rhs = np.einsum("...ab,...sb->...sa", G, op.apply(psi[None], M, prof)[0])
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


@pytest.mark.parametrize(
    "kind,alpha0,src",
    [("exp_t", 0.4, (0, 0, 0, 0)), ("cosh_t", 0.5, (1, 0, 1, 0)), ("cosh_4d", 0.3, (2, 1, 0, 1))],
)
def test_similarity_transform_dense(kind, alpha0, src):
    dims = (4, 2, 2, 2)
    op = oracle.WilsonClover(li.su3_links(dims, 0.5, seed=2), dims, 1.7, -1)
    M = 0.3
    Dp = oracle.dense_matrix(op, M, (kind, alpha0, src))
    D = oracle.dense_matrix(op, M)
    al = oracle.profile_alpha(kind, alpha0, dims, src)
    a = np.repeat(oracle.site_alpha(al, dims).reshape(-1), 12)
    want = (a[:, None] * D) / a[None, :]
    assert np.abs(Dp - want).max() < 1e-14 * np.abs(want).max() * 10
    if kind != "none":
        assert np.abs(Dp - D).max() > 1e-3  # the transform is not trivial


def test_forward_hop_coefficient_orientation():
    """Coefficient of U_mu(x) psi'(x+mu) is -1/2 alpha_B(x)/alpha_B(x+1) (1-gamma_mu)."""
    dims = (5, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, 0.0, -1)
    g = oracle.gammas()
    kind, alpha0, src = "cosh_4d", 0.3, (1, 2, 3, 0)
    al = oracle.profile_alpha(kind, alpha0, dims, src)
    for mu in range(4):
        for x_mu in (0, 1, dims[mu] - 1):
            c = [1, 1, 1, 1]
            c[mu] = x_mu
            cp = list(c)
            cp[mu] = (x_mu + 1) % dims[mu]
            psi = np.zeros(oracle.array_shape(dims) + (4, 3), complex)
            psi[cp[0], cp[3], cp[2], cp[1], :, 0] = [1, 2, 3, 4]
            out = op.apply(psi[None], 0.0, (kind, alpha0, src))[0]
            got = out[c[0], c[3], c[2], c[1], :, 0]
            sign = -1.0 if (mu == 0 and x_mu == dims[0] - 1) else 1.0
            coef = sign * al[mu][x_mu] / al[mu][cp[mu]]
            want = -0.5 * coef * (np.eye(4) - g[mu]) @ np.array([1, 2, 3, 4])
            assert np.abs(got - want).max() < 1e-14
