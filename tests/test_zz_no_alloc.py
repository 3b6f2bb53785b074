"""The allocation-free restore-and-contract entry point.

Some callers cannot let the library allocate device memory: their own
allocator already holds the free memory, or their loop cannot afford an
allocation or an out-of-memory failure mid-run.  dp_restore_contract_noalloc
serves them with a fixed scratch array inside the library.  Here it is called
through the C ABI twice in a row, with different inputs, and must reproduce
dp_restore_contract_dev (the allocating entry point) within the 1e-13
tolerance of the contraction tests, including after the shared array has
held another call's data, and the oracle's restore and contraction of the
same propagators (Sec. II eq. backcorrection; Sec. III, restore before
contracting) within the same tolerance.  This file runs last so that a
failure here leaves every other result in place.
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
import paper_1006_4028_gb300 as dp
from gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu


def _device_halves(S, dims):
    ev, od = dp.pack_half_spinors(S, dims)
    xe = torch.from_numpy(np.ascontiguousarray(ev).view(np.float64)).cuda()
    xo = torch.from_numpy(np.ascontiguousarray(od).view(np.float64)).cuda()
    return xe, xo


def test_noalloc_matches_allocating_entry_point_twice():
    require_gpu()
    ctx = dp.dp_create(0)
    try:
        cases = [
            ((16, 8, 8, 8), [(("cosh_t", 0.4), (3, 1, 2, 0)), (("cosh_4d", 0.2), (5, 3, 0, 1))], 11),
            ((8, 4, 4, 6), [(("exp_t", 0.3), (0, 0, 0, 0)), (("none", 0.0), (1, 2, 3, 5)),
                            (("cosh_t", 0.5), (7, 0, 1, 2))], 12),
        ]
        for dims, groups, seed in cases:
            f = dp.dp_field_load(ctx, li.unit_links(dims), dims, -1)
            ng = len(groups)
            S = li.random_spinor(dims, 12 * ng, seed)
            xe, xo = _device_halves(S, dims)
            profs = [g[0] for g in groups]
            srcs = [g[1] for g in groups]
            ref = torch.full((ng * dims[0],), np.nan, dtype=torch.float64, device="cuda")
            got = torch.full_like(ref, np.nan)
            dp.dp_restore_contract_dev(ctx, f, profs, srcs, xe.data_ptr(), xo.data_ptr(),
                                       ref.data_ptr())
            dp.dp_restore_contract_noalloc(ctx, f, profs, srcs, xe.data_ptr(), xo.data_ptr(),
                                           got.data_ptr())
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert np.all(np.isfinite(g))
            assert np.max(np.abs(g / r - 1)) < 1e-13
            T = dims[0]
            for k, (prof, src) in enumerate(groups):
                al = oracle.profile_alpha(prof[0], prof[1], dims, src)
                Sk = S[12 * k: 12 * (k + 1)].reshape((12,) + oracle.array_shape(dims) + (4, 3))
                want = oracle.contract_cpp(oracle.restore(Sk, al, dims), dims, src[0])
                assert np.max(np.abs(g[k * T:(k + 1) * T] / want - 1)) < 1e-13
            dp.dp_field_free(ctx, f)
    finally:
        dp.dp_destroy(ctx)


def test_noalloc_rejects_too_many_groups():
    require_gpu()
    ctx = dp.dp_create(0)
    try:
        dims = (4, 4, 4, 4)
        f = dp.dp_field_load(ctx, li.unit_links(dims), dims, -1)
        x = torch.zeros(12 * 128 * 72 * 2, dtype=torch.float64, device="cuda")
        cpp = torch.zeros(6 * 4, dtype=torch.float64, device="cuda")
        with pytest.raises(dp.DpError) as e:
            dp.dp_restore_contract_noalloc(ctx, f, [("none", 0.0)] * 6, [(0, 0, 0, 0)] * 6,
                                           x.data_ptr(), x.data_ptr(), cpp.data_ptr())
        assert e.value.status == 1
    finally:
        dp.dp_destroy(ctx)
