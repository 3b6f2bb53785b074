"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds input generation only: gauge links, random spinors and
random gauge transformations.  None of the method's arithmetic (Dirac
operator, preconditioning profile, solver, restore, contraction) lives here,
so the oracle and the GPU library can both draw the same inputs without
sharing any of the computation that is being checked.

Conventions (shared by both sides because they are the input format):

* ``dims = (T, Lx, Ly, Lz)``; lexicographic site index
  ``i = ((t*Lz + z)*Ly + y)*Lx + x``.
* links: complex128 array of shape ``(T, Lz, Ly, Lx, 4, 3, 3)``; direction
  ``mu = 0`` is time, ``1, 2, 3`` are x, y, z; ``U[..., mu, a, b]`` is row a,
  column b of ``U_mu(x)``.
* spinors: complex128 array of shape ``(nrhs, T, Lz, Ly, Lx, 4, 3)`` (spin,
  colour).

Synthetic links follow the recipe of the interacting workloads: an su(3)
element ``H = sum_a c_a lambda_a / 2`` with ``c_a ~ N(0, 1)`` (the eight
Gell-Mann matrices), ``U = exp(i eps H)`` through a Hermitian
eigen-decomposition, then re-unitarised (Gram-Schmidt on rows 0 and 1, row 2
set to ``conj(row0 x row1)`` so that ``det U = 1``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "lattice_shape",
    "unit_links",
    "su3_links",
    "random_spinor",
    "haar_su3",
    "random_gauge_transform",
    "abelian_flux_links",
]


def lattice_shape(dims):
    """Array shape ``(T, Lz, Ly, Lx)`` of a lattice with ``dims = (T, Lx, Ly, Lz)``."""
    T, Lx, Ly, Lz = (int(d) for d in dims)
    return (T, Lz, Ly, Lx)


def gell_mann():
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _reunitarise(U):
    """Gram-Schmidt rows 0 and 1, row 2 = conj(row0 x row1): det = 1."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def unit_links(dims):
    """Free field: every link is the 3x3 identity."""
    shp = lattice_shape(dims) + (4, 3, 3)
    U = np.zeros(shp, dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def su3_links(dims, eps, seed):
    """Synthetic SU(3) links ``U = exp(i eps H)``, ``H = sum_a c_a lambda_a/2``.

    The coefficients are drawn as one ``N(0, 1)`` array of shape
    ``(T, Lz, Ly, Lx, 4, 8)`` from ``numpy.random.default_rng(seed)``.
    """
    shp = lattice_shape(dims) + (4,)
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(shp + (8,))
    H = np.einsum("...a,aij->...ij", c, gell_mann() / 2)
    w, V = np.linalg.eigh(H)
    U = np.einsum("...ij,...j,...kj->...ik", V, np.exp(1j * eps * w), np.conj(V))
    return _reunitarise(U)


def random_spinor(dims, nrhs, seed):
    """Gaussian complex spinors, real and imaginary parts ``N(0, 1)``."""
    shp = (int(nrhs),) + lattice_shape(dims) + (4, 3)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    return re + 1j * im


def haar_su3(n, seed):
    """``n`` Haar-random SU(3) matrices (QR of a complex Gaussian, phase-fixed)."""
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    Q[:, :, 2] = Q[:, :, 2] / det[:, None]
    return Q


def random_gauge_transform(dims, seed):
    """A Haar-random ``G(x)`` per site, shape ``(T, Lz, Ly, Lx, 3, 3)``."""
    shp = lattice_shape(dims)
    return haar_su3(int(np.prod(shp)), seed).reshape(shp + (3, 3))


def abelian_flux_links(dims, mu, nu, n_flux, charges=(1.0, -1.0, 0.0)):
    """Links carrying a constant abelian field strength in the (mu, nu) plane.

    ``U_nu(x) = exp(i F x_mu Q)`` and, on the last ``x_mu`` layer,
    ``U_mu(x) = exp(-i F L_mu x_nu Q)``, all other links 1, with
    ``F = 2 pi n_flux / (L_mu L_nu)`` and ``Q = diag(charges)`` traceless.
    Every plaquette in the (mu, nu) plane then equals ``exp(i F Q)`` (the
    flux is quantised so the torus closes), and every other plaquette is 1.
    """
    T, Lx, Ly, Lz = (int(d) for d in dims)
    L = {0: T, 1: Lx, 2: Ly, 3: Lz}
    axis = {0: 0, 1: 3, 2: 2, 3: 1}  # direction -> array axis of (T, Lz, Ly, Lx)
    F = 2 * np.pi * n_flux / (L[mu] * L[nu])
    q = np.asarray(charges, dtype=np.float64)
    U = unit_links(dims)
    shp = lattice_shape(dims)
    coords = np.indices(shp)
    xmu = coords[axis[mu]]
    xnu = coords[axis[nu]]
    ph_nu = F * xmu
    ph_mu = np.where(xmu == L[mu] - 1, -F * L[mu] * xnu, 0.0)
    for a in range(3):
        U[..., nu, a, a] = np.exp(1j * ph_nu * q[a])
        U[..., mu, a, a] = np.exp(1j * ph_mu * q[a])
    return U, F
