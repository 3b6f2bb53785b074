"""Host logic of the benchmark: the serving mix's profiles and fields, the
tune cache.  No GPU."""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

def test_serving_mix_profiles():
    """Heavy requests (M >= 0.3) take cosh-t alpha0 = 0.4 (Sec. II eq.
    pbcalpha), light ones the four-dimensional cosh-4d alpha0 = 0.2 (Sec. III
    eq. betaa)."""
    assert bench.c5_profile(0.3) == ("cosh_t", 0.4)
    assert bench.c5_profile(0.8) == ("cosh_t", 0.4)
    assert bench.c5_profile(0.29) == ("cosh_4d", 0.2)
    assert bench.c5_profile(0.01) == ("cosh_4d", 0.2)
    assert [d for d, _, _ in bench.C5_FIELDS] == [(16, 8, 8, 8), (32, 16, 16, 16),
                                                  (48, 24, 24, 24), (64, 32, 32, 32)]


def test_tune_cache_round_trip(tmp_path):
    path = str(tmp_path / "state" / "tunecache.json")
    assert bench.load_tune_cache(path) == {}
    bench.save_tune_cache(path, {"48x24x24x24 mixed_fp32_n12": [128, 2, 6]})
    assert bench.load_tune_cache(path) == {"48x24x24x24 mixed_fp32_n12": [128, 2, 6]}
    with open(path, "w") as fh:
        fh.write("{not json")
    assert bench.load_tune_cache(path) == {}
    bench.save_tune_cache("none", {"x": [1, 2, 3]})
    assert not os.path.exists("none")
    assert bench.load_tune_cache("none") == {}


def test_oracle_operator_timing_reports_rate():
    """The per-workload CPU baseline helper: one timed full-lattice (D+M)
    application of the oracle on a small lattice, with its rate and the
    operator it built (reused by the workloads' timed oracle solves)."""
    import lattice_inputs as li

    dims = (4, 4, 4, 4)
    op, rate = bench.oracle_dslash_rate(li.su3_links(dims, 0.3, 1), dims, 1.7, 0.5,
                                        ("cosh_t", 0.4), reps=1)
    assert rate["kind"] == "oracle" and rate["cores"] >= 1
    assert rate["ms_per_application"] > 0
    V = 4 ** 4
    assert math.isclose(rate["sites_per_s"], V / (rate["ms_per_application"] / 1e3), rel_tol=1e-9)
    assert math.isclose(rate["algorithmic_gbs"],
                        V * 192 * 8 / (rate["ms_per_application"] / 1e3) / 1e9, rel_tol=1e-9)
    assert op.dims == dims
