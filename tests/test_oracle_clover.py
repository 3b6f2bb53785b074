"""Pins of the oracle's clover term c_sw (i/4) sum sigma_{mu nu} Fhat_{mu nu}.

* Fhat vanishes at U = 1;
* on a constant abelian field strength F in one plane, every leaf equals
  exp(i F Q), so Fhat = i sin(F Q) exactly (leaf orientation, the 1/8
  normalisation and the Q - Q^dag combination are all tested);
* Fhat is anti-Hermitian and gauge covariant; the clover term is Hermitian.
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle

AX = {0: 0, 1: 3, 2: 2, 3: 1}


def gauge_transform(U, G):
    """U^G_mu(x) = G(x) U_mu(x) G(x+mu)^dag."""
    out = np.empty_like(U)
    for mu in range(4):
        Gp = np.roll(G, -1, axis=AX[mu])
        out[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(Gp, -1, -2))
    return out


def test_clover_vanishes_free_field():
    dims = (4, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=1.9)
    assert np.abs(op.F).max() == 0.0


@pytest.mark.parametrize("plane", [(0, 1), (1, 2), (3, 0), (2, 3)])
def test_abelian_constant_field_closed_form(plane):
    mu, nu = plane
    dims = (6, 4, 6, 4)
    charges = (1.0, -1.0, 0.0)
    U, F = li.abelian_flux_links(dims, mu, nu, n_flux=1, charges=charges)
    op = oracle.WilsonClover(U, dims, csw=1.3)
    Fh = op.F.reshape(oracle.array_shape(dims) + (4, 4, 3, 3))
    want = np.diag(1j * np.sin(F * np.asarray(charges)))
    for a in range(4):
        for b in range(4):
            blk = Fh[..., a, b, :, :]
            if (a, b) == (mu, nu):
                ref = want
            elif (a, b) == (nu, mu):
                ref = -want
            else:
                ref = np.zeros((3, 3))
            assert np.abs(blk - ref).max() < 1e-14
    # clover term on that background: c_sw (i/2) sigma_{mu nu} Fhat_{mu nu}
    #   = -(c_sw/2) sin(F q_a) sigma_{mu nu}  on colour a
    psi = li.random_spinor(dims, 1, seed=5)
    got = op.clover(psi)
    sg = oracle.sigmas()[mu, nu]
    q = np.asarray(charges)
    ref = np.einsum("st,...tc->...sc", sg, psi) * (-(1.3 / 2) * np.sin(F * q))
    assert np.abs(got - ref).max() < 1e-14


def test_field_strength_antihermitian_and_covariant():
    dims = (4, 4, 4, 4)
    U = li.su3_links(dims, 0.5, seed=3)
    op = oracle.WilsonClover(U, dims, csw=1.0)
    F = op.F
    assert np.abs(F + np.conj(np.swapaxes(F, -1, -2))).max() < 1e-14
    assert np.abs(F + np.swapaxes(F, 1, 2)).max() < 1e-14  # Fhat_nu,mu = -Fhat_mu,nu
    G = li.random_gauge_transform(dims, seed=9)
    opG = oracle.WilsonClover(gauge_transform(U, G), dims, csw=1.0)
    Gs = G.reshape(-1, 1, 1, 3, 3)
    want = Gs @ F @ np.conj(np.swapaxes(Gs, -1, -2))
    assert np.abs(opG.F - want).max() < 1e-13


def test_clover_term_hermitian():
    dims = (4, 4, 4, 4)
    U = li.su3_links(dims, 0.4, seed=4)
    op = oracle.WilsonClover(U, dims, csw=1.7)
    phi = li.random_spinor(dims, 1, 1)
    psi = li.random_spinor(dims, 1, 2)
    lhs = np.vdot(phi, op.clover(psi))
    rhs = np.vdot(op.clover(phi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the clover term commutes with gamma_5 (it is chirally block diagonal)
    g5 = oracle.gamma5()
    a = op.clover(np.einsum("st,...tc->...sc", g5, psi))
    b = np.einsum("st,...tc->...sc", g5, op.clover(psi))
    assert np.abs(a - b).max() < 1e-13


def test_operator_is_diagonal_plus_hop_plus_clover():
    """(D+M) = (4+M) + hopping term + clover term, the clover term applied from
    its per-site matrix form inside the operator."""
    dims = (4, 4, 4, 4)
    op = oracle.WilsonClover(li.su3_links(dims, 0.4, seed=6), dims, csw=1.9)
    psi = li.random_spinor(dims, 2, 3)
    M = 0.27
    prof = ("cosh_4d", 0.3, (1, 2, 3, 0))
    lhs = op.apply(psi, M, prof)
    rhs = (4 + M) * psi + op.hop(psi, prof) + op.clover(psi)
    assert np.abs(lhs - rhs).max() < 1e-13
