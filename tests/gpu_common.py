"""Shared helpers of the GPU tests (imported by tests marked `gpu` only)."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def per_site_rel(got, ref):
    """max over sites of |got(x) - ref(x)|_2 / |ref(x)|_2 (spin-colour norm)."""
    g = np.asarray(got).reshape(-1, 12)
    r = np.asarray(ref).reshape(-1, 12)
    num = np.linalg.norm(g - r, axis=1)
    den = np.linalg.norm(r, axis=1)
    return float(np.max(num / den))


def slice_rel(got, ref, upto):
    g = np.asarray(got)[: upto + 1]
    r = np.asarray(ref)[: upto + 1]
    return float(np.max(np.abs(g / r - 1)))


def field(dims, eps, seed):
    return li.unit_links(dims) if eps == 0 else li.su3_links(dims, eps, seed)
