"""Pins of the oracle's per-time-slice residual (``oracle.slice_residuals``).

rho(y0) = |[eta - (D+M) S]_t| / |S_t| is the quantity the library's outer
loop drives below its per-slice target so that C_PP stays accurate on the far
slices (the paper's error argument, Sec. II).  Pinned by:

* the exact free propagator (momentum space) gives rho at rounding level on
  every slice;
* a perturbation delta planted on one slice t0 of that propagator leaves
  every slice beyond t0 +- 1 untouched, and on t0 + 1 and t0 - 1 the residual
  is the time hop of delta alone: -1/2 (1 +- gamma_0) delta, i.e. the chiral
  projections P+- delta with P+- = (1 +- gamma_0)/2 (U = 1), so
  rho(t0 + 1) = |P+ delta| / |S_{t0+1}| and rho(t0 - 1) = |P- delta| / |S_{t0-1}|.
"""
import numpy as np

import lattice_inputs as li
import oracle


def _free_point_solution(dims, M):
    Sf = oracle.free_propagator(dims, M, -1)  # (T, Lz, Ly, Lx, sink spin, source spin)
    S = np.zeros((12,) + oracle.array_shape(dims) + (4, 3), complex)
    for k in range(12):
        S[k, ..., :, k % 3] = Sf[..., :, k // 3]
    return S


def test_exact_free_solution_has_rounding_level_slice_residuals():
    dims, M = (12, 4, 4, 4), 0.5
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=1.7, bc_t=-1)
    S = _free_point_solution(dims, M)
    eta = oracle.point_sources(dims, (0, 0, 0, 0))
    rho = oracle.slice_residuals(op, M, S, eta, 0)
    assert rho.shape == (12,)
    assert rho.max() < 1e-12


def test_planted_slice_error_is_localised_with_the_projector_residuals():
    dims, M, t0 = (12, 4, 4, 4), 0.5, 6
    op = oracle.WilsonClover(li.unit_links(dims), dims, csw=1.7, bc_t=-1)
    S = _free_point_solution(dims, M)
    eta = oracle.point_sources(dims, (0, 0, 0, 0))
    rng = np.random.default_rng(3)
    delta = np.zeros_like(S)
    shape = delta[:, t0].shape
    delta[:, t0] = 1e-3 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    rho = oracle.slice_residuals(op, M, S + delta, eta, 0)
    far = [t for t in range(dims[0]) if abs(t - t0) > 1]
    assert rho[far].max() < 1e-12
    g0 = oracle.gammas()[0]
    Pp = 0.5 * (np.eye(4) + g0)
    Pm = 0.5 * (np.eye(4) - g0)
    d = delta[:, t0]
    nPp = np.linalg.norm(np.einsum("st,...tc->...sc", Pp, d))
    nPm = np.linalg.norm(np.einsum("st,...tc->...sc", Pm, d))
    Sp1 = np.linalg.norm(S[:, t0 + 1])
    Sm1 = np.linalg.norm(S[:, t0 - 1])
    assert abs(rho[t0 + 1] / (nPp / Sp1) - 1) < 1e-9
    assert abs(rho[t0 - 1] / (nPm / Sm1) - 1) < 1e-9
    # relative indexing: the same values rotated when the source slice moves
    rho2 = oracle.slice_residuals(op, M, S + delta, eta, 4)
    assert np.allclose(rho2, np.roll(rho, -4), rtol=0, atol=0)
