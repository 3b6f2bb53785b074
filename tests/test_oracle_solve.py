"""Pins of the oracle's solve / restore / contract pipeline.

* BiCGStab against a dense LU solve (LAPACK) on 4^4, with and without a profile;
* the restored preconditioned C_PP equals the unpreconditioned one at tight
  residue, for every profile kind and alpha0 (exact similarity transform,
  Sec. II; restoration eq. backcorrection and Sec. III eq. redefa);
* C_PP is gauge invariant;
* the heavy-quark effect of Sec. II: at a loose residue the unpreconditioned
  far slices go wrong while the preconditioned-and-restored ones stay right.
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from test_oracle_clover import gauge_transform


@pytest.mark.parametrize("profile", [None, ("cosh_4d", 0.3, (1, 0, 2, 3))])
def test_bicgstab_matches_dense_lu_4x4x4x4(profile):
    dims = (4, 4, 4, 4)
    op = oracle.WilsonClover(li.su3_links(dims, 0.4, seed=5), dims, 1.7, -1)
    M = 0.3
    A = oracle.dense_matrix(op, M, profile)
    B = li.random_spinor(dims, 3, seed=6)
    X_lu = np.linalg.solve(A, B.reshape(3, -1).T).T
    X, iters, rel, ok = op.solve(B, M, profile, tol=1e-13)
    assert ok and rel.max() < 1e-13
    err = np.abs(X.reshape(3, -1) - X_lu).max() / np.abs(X_lu).max()
    assert err < 1e-11


def _interacting(dims=(12, 4, 4, 4), eps=0.3, seed=1, csw=1.7):
    return oracle.WilsonClover(li.su3_links(dims, eps, seed=seed), dims, csw, -1)


def test_restored_equals_unpreconditioned_and_alpha0_independent():
    op = _interacting()
    M, src = 0.5, (3, 1, 2, 0)
    ref, _, info = oracle.solve_point(op, M, "none", 0.0, src, tol=1e-13)
    assert info["converged"]
    for kind, a0 in [("cosh_t", 0.3), ("cosh_t", 0.5), ("exp_t", 0.4), ("cosh_4d", 0.2)]:
        cpp, _, info = oracle.solve_point(op, M, kind, a0, src, tol=1e-13)
        assert info["converged"]
        assert np.abs(cpp / ref - 1).max() < 1e-10, (kind, a0)


def test_cpp_gauge_invariant():
    dims = (8, 4, 4, 4)
    U = li.su3_links(dims, 0.4, seed=3)
    G = li.random_gauge_transform(dims, seed=4)
    src = (2, 1, 0, 3)
    a, _, _ = oracle.solve_point(oracle.WilsonClover(U, dims, 1.7), 0.4, "cosh_t", 0.4, src)
    b, _, _ = oracle.solve_point(oracle.WilsonClover(gauge_transform(U, G), dims, 1.7),
                                 0.4, "cosh_t", 0.4, src)
    assert np.abs(b / a - 1).max() < 1e-10


@pytest.mark.slow
def test_heavy_quark_loose_residue_effect():
    """Free heavy quark, T = 48: r = 1e-6 unpreconditioned drifts on the far
    slices; preconditioned (cosh, alpha0 = 0.4) at r = 1e-6 stays accurate."""
    dims = (48, 4, 4, 4)
    op = oracle.WilsonClover(li.unit_links(dims), dims, 0.0, -1)
    M = 0.5
    exact = oracle.free_cpp(dims, M)
    loose, _, _ = oracle.solve_point(op, M, "none", 0.0, (0, 0, 0, 0), tol=1e-6)
    prec, _, _ = oracle.solve_point(op, M, "cosh_t", 0.4, (0, 0, 0, 0), tol=1e-6)
    e_loose = np.abs(loose / exact - 1)[: dims[0] // 2 + 1]
    e_prec = np.abs(prec / exact - 1)[: dims[0] // 2 + 1]
    assert e_loose.max() > 1e-2
    assert e_prec.max() < 1e-4
    # the loose-residue error grows with distance from the source
    assert e_loose[-1] > 100 * e_loose[:4].max()
