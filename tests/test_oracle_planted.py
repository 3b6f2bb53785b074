"""Planted mistakes: each plausible error in the oracle must fail a pin.

Mistakes are planted in the oracle on the CPU (monkeypatching its Python
layer); nothing here touches the GPU library.
"""
import numpy as np

import lattice_inputs as li
import oracle


def test_wrong_time_boundary_sign_fails_free_pin():
    dims = (8, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, 0.0, bc_t=+1)  # planted
    cpp, _, _ = oracle.solve_point(op, 0.5, "none", 0.0, (0, 0, 0, 0), tol=1e-13)
    exact = oracle.free_cpp(dims, 0.5, bc_t=-1)
    assert np.abs(cpp / exact - 1).max() > 1e-3


def test_flipped_gamma_fails_plane_wave_pin(monkeypatch):
    good = oracle.gammas()

    def bad():
        g = good.copy()
        g[0] = -g[0]  # planted: wrong sign of gamma_0
        return g

    dims = (6, 4, 4, 4)
    monkeypatch.setattr(oracle, "gammas", bad)
    op = oracle.WilsonClover(li.unit_links(dims), dims, 0.0, -1)
    monkeypatch.setattr(oracle, "gammas", lambda: good)
    t, x, y, z = oracle.site_coords(dims)
    p = [2 * np.pi * 1.5 / 6, 2 * np.pi / 4, 0.0, 0.0]
    chi = np.arange(12).reshape(4, 3) + 1j
    psi = np.exp(1j * (p[0] * t + p[1] * x))[..., None, None] * chi
    got = op.apply(psi[None], 0.3)[0]
    want = np.einsum("st,...tc->...sc", oracle.free_momentum_operator(p, 0.3), psi)
    assert np.abs(got - want).max() > 1e-2


def test_reversed_profile_orientation_fails_similarity_pin(monkeypatch):
    dims = (4, 2, 2, 2)
    op = oracle.WilsonClover(li.su3_links(dims, 0.5, seed=2), dims, 1.7, -1)
    kind, a0, src = "cosh_t", 0.5, (1, 0, 0, 0)
    al = oracle.profile_alpha(kind, a0, dims, src)
    good_tables = oracle.hop_tables

    def bad(alphas, d, bc):
        return good_tables([1.0 / a for a in alphas], d, bc)  # planted: alpha_P used as alpha_B

    monkeypatch.setattr(oracle, "hop_tables", bad)
    Dp = oracle.dense_matrix(op, 0.3, (kind, a0, src))
    monkeypatch.setattr(oracle, "hop_tables", good_tables)
    D = oracle.dense_matrix(op, 0.3)
    a = np.repeat(oracle.site_alpha(al, dims).reshape(-1), 12)
    want = (a[:, None] * D) / a[None, :]
    assert np.abs(Dp - want).max() > 1e-2


def test_restore_by_multiplication_fails_restore_pin(monkeypatch):
    dims = (8, 4, 4, 4)
    op = oracle.WilsonClover(li.su3_links(dims, 0.3, seed=1), dims, 1.7, -1)
    ref, _, _ = oracle.solve_point(op, 0.5, "none", 0.0, (0, 0, 0, 0))
    good = oracle.restore

    def bad(Sp, alphas, d):
        return good(Sp, [1.0 / a for a in alphas], d)  # planted: S = alpha_B S'

    monkeypatch.setattr(oracle, "restore", bad)
    cpp, _, _ = oracle.solve_point(op, 0.5, "cosh_t", 0.4, (0, 0, 0, 0))
    assert np.abs(cpp / ref - 1).max() > 1e-2


def test_clover_normalisation_error_fails_abelian_pin(monkeypatch):
    good = oracle.sigmas
    monkeypatch.setattr(oracle, "sigmas", lambda: 2 * good())  # planted: factor 2
    dims = (6, 4, 6, 4)
    U, F = li.abelian_flux_links(dims, 1, 2, 1)
    op = oracle.WilsonClover(U, dims, 1.3)
    monkeypatch.setattr(oracle, "sigmas", good)
    psi = li.random_spinor(dims, 1, seed=5)
    got = op.clover(psi)
    q = np.array([1.0, -1.0, 0.0])
    ref = np.einsum("st,...tc->...sc", good()[1, 2], psi) * (-(1.3 / 2) * np.sin(F * q))
    assert np.abs(got - ref).max() > 1e-2
