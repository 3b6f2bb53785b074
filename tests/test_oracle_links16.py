"""Pins of the oracle's 16-bit link storage (rows 0 and 1 in FP16 / BF16 with
one FP32 scale per link, row 2 rebuilt from unitarity and det U = 1 of the
SU(3) links, Sec. I).

Independent checks: torch's own float32 -> bfloat16 / float16 conversions,
hand-worked ties, exactly representable links, the rounding-error bound of
each format, and a non-SU(3) link whose rebuilt row differs from the stored
one in a known way.
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle


def test_bf16_ties_and_values():
    x = np.array([1 + 2**-8, 1 + 3 * 2**-8, 1 + 2**-8 + 2**-20, -(1 + 2**-8), 3.0, 0.0, 2**-130],
                 np.float32)
    want = np.array([1.0, 1 + 2**-6, 1 + 2**-7, -1.0, 3.0, 0.0, 2**-130], np.float64)
    np.testing.assert_array_equal(oracle.round_bf16(x).astype(np.float64), want)


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x), ref)


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_unit_links_are_stored_exactly(kind):
    U = li.unit_links((2, 2, 2, 2))
    np.testing.assert_array_equal(oracle.stored_links16(U, kind), U)


@pytest.mark.parametrize("kind,half_ulp", [("fp16", 2.0**-11), ("bf16", 2.0**-8)])
def test_rounding_bound_and_representable(kind, half_ulp):
    """Each stored real of rows 0, 1 is s*q with q in the 16-bit format and
    |s q - u| <= s (half an ulp at 1 + FP32 rounding); row 2 then deviates
    from the exact row 2 by at most twice the row-error norm."""
    torch = pytest.importorskip("torch")
    dims = (4, 4, 2, 2)
    U = li.su3_links(dims, 0.6, 9)
    S = oracle.stored_links16(U, kind)
    rows = U[..., :2, :]
    s = np.maximum(np.abs(rows.real), np.abs(rows.imag)).max(axis=(-2, -1)).astype(np.float32)
    s = s.astype(np.float64)[..., None, None]
    q = np.concatenate([S[..., :2, :].real / s, S[..., :2, :].imag / s])
    tdt = torch.float16 if kind == "fp16" else torch.bfloat16
    back = torch.from_numpy(q.astype(np.float32)).to(tdt).to(torch.float64).numpy()
    np.testing.assert_array_equal(back, q)
    d = S[..., :2, :] - rows
    bound = s * (half_ulp + 2.0**-24)
    assert np.all(np.abs(d.real) <= bound) and np.all(np.abs(d.imag) <= bound)
    row_err = np.sqrt(6) * bound[..., 0, 0]
    e2 = np.abs(S[..., 2, :] - U[..., 2, :]).max(axis=-1)
    assert np.all(e2 <= 2.05 * row_err)
    # the largest deviation is of the order of the format's resolution
    assert np.abs(d).max() > 0.1 * half_ulp * s.min()


def test_row2_is_rebuilt_not_stored():
    """U = i * identity (unitary, det = -i): rows 0, 1 are stored exactly and
    the rebuilt row 2 is conj((i e0) x (i e1)) = conj(-e2) = -e2, not i e2."""
    U = li.unit_links((2, 2, 2, 2)) * 1j
    for kind in ("fp16", "bf16"):
        S = oracle.stored_links16(U, kind)
        np.testing.assert_array_equal(S[..., :2, :], U[..., :2, :])
        np.testing.assert_array_equal(S[..., 2, :], -li.unit_links((2, 2, 2, 2))[..., 2, :])
