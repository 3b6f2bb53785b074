"""Orientation pins of the oracle's profiles (``oracle.profile_alpha``).

The restored result does not depend on the profile, so the profile's
direction is invisible to every restore-based pin; it is fixed here by what
the paper says each profile is for, measured on the exact momentum-space
free propagator S (independent of the oracle's operator and solver):

* heavy quark, Sec. II eq. (pbcalpha): the time profile is chosen so that the
  preconditioned propagator S' = alpha_B S is roughly flat; with alpha0 at the
  free pole energy ln(1+M) its slice norms stay within a small factor of each
  other while those of S fall by many decades;
* light quark, Sec. III eq. (betaa): the four-dimensional profile grows away
  from the centre of the lattice seen from the source, so it makes S'
  steeper than S (the far/near ratio shrinks);
* the SF form of Sec. II (exp profile): alpha_B grows with the distance from
  the source, and the time hop across the antiperiodic seam carries the ratio
  of the two slices' actual values, alpha_B(T-1)/alpha_B(0) = e^{alpha0 (T-1)},
  times the boundary sign (eq. redeftbc).
"""
import numpy as np

import oracle

DIMS = (32, 4, 4, 4)
M = 0.5


def _slice_norms(S):
    return np.sqrt(np.sum(np.abs(S) ** 2, axis=tuple(range(1, S.ndim))))


def _free():
    return oracle.free_propagator(DIMS, M, -1)  # (T, Lz, Ly, Lx, 4, 4)


def _primed(kind, alpha0):
    al = oracle.profile_alpha(kind, alpha0, DIMS)
    a = oracle.site_alpha(al, DIMS)
    return a[..., None, None] * _free()


def test_heavy_cosh_profile_flattens_the_propagator():
    n = _slice_norms(_free())
    npr = _slice_norms(_primed("cosh_t", np.log(1 + M)))
    T = DIMS[0]
    fall = n[T // 2] / n[1]
    fall_p = npr[T // 2] / npr[1]
    assert fall < 1e-2              # the propagator itself falls by decades
    assert 0.1 < fall_p < 10.0      # the preconditioned one is roughly flat
    assert npr.max() / npr.min() < 1e2


def test_light_cosh4d_profile_steepens_the_propagator():
    n = _slice_norms(_free())
    npr = _slice_norms(_primed("cosh_4d", 0.2))
    T = DIMS[0]
    assert npr[T // 2] / npr[0] < 0.5 * (n[T // 2] / n[0])
    # and alpha_B itself is largest at the source, smallest half a lattice away
    al = oracle.profile_alpha("cosh_4d", 0.2, DIMS)
    for mu, L in enumerate(DIMS):
        assert np.argmax(al[mu]) == 0 and np.argmin(al[mu]) == L // 2


def test_exp_profile_grows_and_carries_the_seam_ratio():
    T, a0 = DIMS[0], 0.3
    al = oracle.profile_alpha("exp_t", a0, DIMS)
    assert np.all(np.diff(al[0]) > 0)
    fwd, bwd, _ = oracle.hop_tables(al, DIMS, -1)
    assert abs(fwd[0, T - 1] / (-np.exp(a0 * (T - 1))) - 1) < 1e-14
    assert abs(bwd[0, 0] / (-np.exp(-a0 * (T - 1))) - 1) < 1e-14
    # bulk hops: forward factor alpha(x)/alpha(x+1) = e^{-alpha0}
    assert np.allclose(fwd[0, : T - 1], np.exp(-a0), rtol=1e-14, atol=0)
