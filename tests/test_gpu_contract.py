"""Restore and contract (Sec. II eq. backcorrection; Sec. III: restore before
contracting) on the GPU against the oracle, for a device-resident S'."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
import paper_1006_4028_gb300 as dp
from gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu

GROUPS = [(("cosh_t", 0.4), (3, 1, 2, 0)), (("cosh_4d", 0.2), (5, 3, 0, 1)),
          (("exp_t", 0.3), (0, 0, 0, 0))]


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    c = dp.dp_create(0)
    yield c
    dp.dp_destroy(c)


def contract_case(ctx, dims, groups, seed):
    f = dp.dp_field_load(ctx, li.unit_links(dims), dims, -1)
    ng = len(groups)
    Sp = li.random_spinor(dims, 12 * ng, seed)
    ev, od = dp.pack_half_spinors(Sp, dims)
    xe = torch.from_numpy(np.ascontiguousarray(ev).view(np.float64)).cuda()
    xo = torch.from_numpy(np.ascontiguousarray(od).view(np.float64)).cuda()
    cpp = torch.full((ng * dims[0],), np.nan, dtype=torch.float64, device="cuda")
    dp.dp_restore_contract_dev(ctx, f, [g[0] for g in groups], [g[1] for g in groups],
                               xe.data_ptr(), xo.data_ptr(), cpp.data_ptr())
    torch.cuda.synchronize()
    got = cpp.cpu().numpy().reshape(ng, dims[0])
    dp.dp_field_free(ctx, f)
    want = []
    for k, (prof, src) in enumerate(groups):
        al = oracle.profile_alpha(prof[0], prof[1], dims, src)
        S = oracle.restore(Sp[12 * k:12 * k + 12], al, dims)
        want.append(oracle.contract_cpp(S, dims, src[0]))
    return got, np.asarray(want)


@pytest.mark.parametrize("dims", [(8, 4, 4, 6), (16, 8, 8, 8)])
def test_restore_contract_matches_oracle(ctx, dims):
    got, want = contract_case(ctx, dims, GROUPS, 3)
    assert np.max(np.abs(got / want - 1)) < 1e-13
