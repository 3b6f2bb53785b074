"""Serving: continuous batching of point-source requests over resident fields.

A request's result must be the same alone and in a mix of concurrent
requests (stated tolerance 1e-6 per slice; the design target is bit
identity, since every per-RHS decision and reduction is independent of the
other slots), and must match the oracle.
"""
import time

import numpy as np
import pytest

import oracle
import paper_1006_4028_gb300 as dp
from gpu_common import field, require_gpu, slice_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    require_gpu()
    c = dp.dp_create(0)
    fields = {}
    for dims, eps, seed in [((8, 4, 4, 4), 0.3, 101), ((12, 4, 4, 6), 0.4, 102)]:
        U = field(dims, eps, seed)
        f = dp.dp_field_load(c, U, dims, -1)
        dp.dp_field_set_csw(c, f, 1.7)
        fields[f] = (dims, oracle.WilsonClover(U, dims, 1.7, -1))
    dp.dp_serve_start(c, 0, 24)
    yield c, fields
    dp.dp_serve_stop(c, True)
    dp.dp_destroy(c)


def test_same_result_alone_and_in_mix(served):
    c, fields = served
    fids = list(fields)
    f0 = fids[0]
    T0 = fields[f0][0][0]
    req = (f0, 0.5, ("cosh_t", 0.4), (1, 2, 3, 0), 1e-10)
    t = dp.dp_submit(c, *req)
    alone, info = dp.dp_wait(c, t, T0, timeout_s=120)
    assert info["status"] == 0
    # a mix on both fields, the same request submitted in the middle
    rng = np.random.default_rng(2024)
    tickets = []
    for k in range(7):
        f = fids[k % 2]
        dims = fields[f][0]
        M = float(rng.uniform(0.01, 0.8))
        prof = ("cosh_t", 0.4) if M >= 0.3 else ("cosh_4d", 0.2)
        src = tuple(int(rng.integers(0, d)) for d in dims)
        tickets.append((dp.dp_submit(c, f, M, prof, src, 1e-10), f, M, prof, src))
        if k == 3:
            same = dp.dp_submit(c, *req)
    mixed, _ = dp.dp_wait(c, same, T0, timeout_s=120)
    assert slice_rel(mixed, alone, T0 // 2) < 1e-6
    np.testing.assert_array_equal(mixed, alone)  # design target: bit identical
    dims0, op0 = fields[f0]
    ref, _, _ = oracle.solve_point(op0, req[1], req[2][0], req[2][1], req[3], tol=1e-13)
    assert slice_rel(alone, ref, T0 // 2) < 1e-6
    for tk, f, M, prof, src in tickets:
        dims, op = fields[f]
        cpp, info = dp.dp_wait(c, tk, dims[0], timeout_s=120)
        assert info["status"] == 0
        ref, _, _ = oracle.solve_point(op, M, prof[0], prof[1], src, tol=1e-13)
        assert slice_rel(cpp, ref, dims[0] // 2) < 1e-6
    st = dp.dp_serve_stats_get(c)
    assert st["completed"] >= 9 and st["p99_ms"] >= st["p50_ms"] > 0


def test_wait_timeout_and_cancel(served):
    c, fields = served
    f = list(fields)[1]
    dims = fields[f][0]
    tks = [dp.dp_submit(c, f, 0.02, ("cosh_4d", 0.2), (0, 0, 0, 0), 1e-10) for _ in range(6)]
    with pytest.raises(dp.DpError) as e:
        dp.dp_wait(c, tks[-1], dims[0], timeout_s=0.0)
    assert e.value.status == 6
    # the last one is still queued behind the running slots: cancel it
    cancelled = False
    try:
        dp.dp_cancel(c, tks[-1])
        cancelled = True
    except dp.DpError:
        pass
    for t in tks[:-1]:
        dp.dp_wait(c, t, dims[0], timeout_s=300)
    if cancelled:
        with pytest.raises(dp.DpError) as e:
            dp.dp_wait(c, tks[-1], dims[0], timeout_s=10)
        assert e.value.status == 7
    else:
        dp.dp_wait(c, tks[-1], dims[0], timeout_s=300)


def test_rejected_when_budget_too_small():
    require_gpu()
    c = dp.dp_create(0)
    dims = (8, 4, 4, 4)
    f = dp.dp_field_load(c, field(dims, 0.3, 1), dims, -1)
    dp.dp_field_set_csw(c, f, 1.7)
    dp.dp_serve_start(c, 1 << 20, 12)  # 1 MiB: no batch can ever fit
    with pytest.raises(dp.DpError) as e:
        dp.dp_submit(c, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-8)
    assert e.value.status == 7
    assert dp.dp_serve_stats_get(c)["rejected"] == 1
    dp.dp_serve_stop(c, False)
    with pytest.raises(dp.DpError):
        dp.dp_submit(c, f, 0.5, ("cosh_t", 0.4), (0, 0, 0, 0), 1e-8)
    dp.dp_destroy(c)


def test_mixed_volumes_overlap_and_match_oracle():
    """Two resident fields of different volumes, requests for both in flight
    at once: each field's batch runs on its own stream and worker, so their
    rounds overlap (the scheduler reports two batches inside a round at the
    same time).  Served results against the oracle: the 32x16^3 multi-mass
    workload's field at the origin source (stored oracle results, one request
    per mass with its own profile), and random 16x8^3 requests against live
    oracle solves; 1e-6 per slice out to T/2."""
    import json
    import os

    require_gpu()
    c = dp.dp_create(0)
    try:
        g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                        "cpp_32x16_multimass.json")))
        dims_l = tuple(g["dims"])
        fl = dp.dp_field_load(c, field(dims_l, g["eps"], g["seed"]), dims_l, g["bc_t"])
        dp.dp_field_set_csw(c, fl, g["csw"])
        dims_s = (16, 8, 8, 8)
        Us = field(dims_s, 0.3, 101)
        fs = dp.dp_field_load(c, Us, dims_s, -1)
        dp.dp_field_set_csw(c, fs, 1.7)
        op_s = oracle.WilsonClover(Us, dims_s, 1.7, -1)
        dp.dp_serve_start(c, 0, 24)
        rng = np.random.default_rng(7)
        big, small = [], []
        for k, m in enumerate(g["masses"]):
            prof = ("cosh_t", 0.4 if m["M"] < 0.65 else 0.5) if m["M"] >= 0.3 else ("cosh_4d", 0.2)
            big.append((dp.dp_submit(c, fl, m["M"], prof, (0, 0, 0, 0), 1e-10), m))
            M = float(rng.uniform(0.05, 0.8))
            prof_s = ("cosh_t", 0.4) if M >= 0.3 else ("cosh_4d", 0.2)
            src = tuple(int(rng.integers(0, d)) for d in dims_s)
            small.append((dp.dp_submit(c, fs, M, prof_s, src, 1e-10), M, prof_s, src))
        for t, m in big:
            cpp, info = dp.dp_wait(c, t, dims_l[0], timeout_s=300, allow=())
            assert slice_rel(cpp, np.asarray(m["cpp"]), dims_l[0] // 2) < 1e-6, m["M"]
        for t, M, prof_s, src in small:
            cpp, info = dp.dp_wait(c, t, dims_s[0], timeout_s=300, allow=())
            ref, _, _ = oracle.solve_point(op_s, M, prof_s[0], prof_s[1], src, tol=1e-13)
            assert slice_rel(cpp, ref, dims_s[0] // 2) < 1e-6, (M, prof_s, src)
        st = dp.dp_serve_stats_get(c)
        assert st["completed"] == 8
        assert st["max_concurrent_batches"] == 2
        dp.dp_serve_stop(c, 1)
    finally:
        dp.dp_destroy(c)


def test_interleaved_submits_while_batches_run():
    """Requests for two fields submitted one by one with short random gaps
    while both fields' workers admit and run rounds (the queue changes under
    them): every request completes, and each result equals the same request
    solved directly through dp_solve_point within 1e-6 per slice."""
    require_gpu()
    c = dp.dp_create(0)
    try:
        specs = [((8, 4, 4, 4), 0.3, 201), ((12, 4, 4, 6), 0.4, 202)]
        fields = []
        for dims, eps, seed in specs:
            f = dp.dp_field_load(c, field(dims, eps, seed), dims, -1)
            dp.dp_field_set_csw(c, f, 1.7)
            fields.append((f, dims))
        dp.dp_serve_start(c, 0, 24)
        rng = np.random.default_rng(11)
        reqs = []
        for k in range(40):
            f, dims = fields[k % 2]
            M = float(rng.uniform(0.05, 0.8))
            prof = ("cosh_t", 0.4) if M >= 0.3 else ("cosh_4d", 0.2)
            src = tuple(int(rng.integers(0, d)) for d in dims)
            reqs.append((dp.dp_submit(c, f, M, prof, src, 1e-10), f, dims, M, prof, src))
            time.sleep(float(rng.uniform(0.0, 0.004)))
        served = []
        for t, f, dims, M, prof, src in reqs:
            cpp, info = dp.dp_wait(c, t, dims[0], timeout_s=300, allow=())
            served.append(cpp)
        st = dp.dp_serve_stats_get(c)
        dp.dp_serve_stop(c, 1)
        assert st["completed"] == 40
        for cpp, (t, f, dims, M, prof, src) in zip(served, reqs):
            ref, _, _ = dp.dp_solve_point(c, f, M, prof, src, 1e-10,
                                          {"prec": "mixed_fp32", "batched": 1}, T=dims[0])
            assert slice_rel(cpp, ref, dims[0] // 2) < 1e-6
    finally:
        dp.dp_destroy(c)


def test_request_admitted_at_a_convergence_check():
    """A request that arrives while its field's batch is inside a round (and
    has free slots) ends the running inner solve at its next convergence
    check and is admitted at once; both results still equal direct solves
    (1e-6 per slice)."""
    require_gpu()
    c = dp.dp_create(0)
    try:
        dims = (48, 24, 24, 24)
        f = dp.dp_field_load(c, field(dims, 0.3, 1), dims, -1)
        dp.dp_field_set_csw(c, f, 1.7)
        dp.dp_serve_start(c, 0, 24)
        reqs = [(0.5, ("cosh_t", 0.4), (0, 0, 0, 0)), (0.6, ("cosh_t", 0.4), (5, 3, 2, 1))]
        yielded = False
        for delay in (0.04, 0.02, 0.06):
            t0 = dp.dp_submit(c, f, *reqs[0], 1e-10)
            time.sleep(delay)  # the first request is inside its first round
            t1 = dp.dp_submit(c, f, *reqs[1], 1e-10)
            out = [dp.dp_wait(c, t, dims[0], timeout_s=300, allow=())[0] for t in (t0, t1)]
            if dp.dp_serve_stats_get(c)["yields"] >= 1:
                yielded = True
                break
        dp.dp_serve_stop(c, 1)
        assert yielded
        for cpp, (M, prof, src) in zip(out, reqs):
            ref, _, _ = dp.dp_solve_point(c, f, M, prof, src, 1e-10,
                                          {"prec": "mixed_fp32", "batched": 1}, T=dims[0])
            assert slice_rel(cpp, ref, dims[0] // 2) < 1e-6
    finally:
        dp.dp_destroy(c)
