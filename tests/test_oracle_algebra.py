"""Pins of the oracle's Dirac algebra (chiral basis, gamma_5 = diag(1,1,-1,-1)).

The paper does not fix a gamma basis; C_PP and the propagator norm are basis
independent.  These tests pin the basis the oracle uses to textbook facts.
"""
import numpy as np

import oracle

PAULI = [np.array([[0, 1], [1, 0]], complex),
         np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex)]


def test_gammas_hermitian_and_clifford():
    g = oracle.gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=0)


def test_gamma5_is_chiral_diagonal():
    g5 = oracle.gamma5()
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)
    for g in oracle.gammas():
        assert np.allclose(g5 @ g + g @ g5, 0, atol=0)


def test_sigma_closed_form_in_chiral_basis():
    """sigma_0k = diag(s_k, -s_k), sigma_jk = -eps_jkl diag(s_l, s_l)."""
    sg = oracle.sigmas()
    Z = np.zeros((2, 2))
    for k in range(1, 4):
        s = PAULI[k - 1]
        assert np.allclose(sg[0, k], np.block([[s, Z], [Z, -s]]), atol=1e-15)
        assert np.allclose(sg[k, 0], -np.block([[s, Z], [Z, -s]]), atol=1e-15)
    eps = {(1, 2): 3, (2, 3): 1, (3, 1): 2}
    for (j, k), l in eps.items():
        s = PAULI[l - 1]
        assert np.allclose(sg[j, k], -np.block([[s, Z], [Z, s]]), atol=1e-15)
        assert np.allclose(sg[k, j], np.block([[s, Z], [Z, s]]), atol=1e-15)
    for mu in range(4):
        assert np.allclose(sg[mu, mu], 0)
        for nu in range(4):
            assert np.allclose(sg[mu, nu], sg[mu, nu].conj().T)
            if mu != nu:
                assert np.allclose(sg[mu, nu] @ sg[mu, nu], np.eye(4))
