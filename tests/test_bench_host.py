"""Host logic of the benchmark's serving client: the profile matched to a
quark's calibrated decay rate, the light-profile residue, the tune cache.
No GPU."""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CAL = ([0.01, 0.4, 0.8], [0.5, 0.78, 1.01])  # decay rates of a 64x32^3 field


def test_matched_profile_sits_below_the_decay_rate():
    for M in (0.01, 0.2, 0.4, 0.6, 0.8):
        kind, a0 = bench.matched_profile(M, CAL, 64)
        E = float(__import__("numpy").interp(M, *CAL))
        assert kind == "cosh_t"
        assert abs(a0 - (E - 10 / 64)) <= 0.025 + 1e-12   # rounded to 0.05
        assert abs(a0 / 0.05 - round(a0 / 0.05)) < 1e-9
    # short lattices allow a larger gap (the error grows like exp(c (E - a0) T))
    assert bench.matched_profile(0.8, CAL, 16)[1] < bench.matched_profile(0.8, CAL, 64)[1]


def test_light_quarks_keep_the_light_profile():
    light = ([0.01, 0.4, 0.8], [0.16, 0.55, 0.86])  # a 16x8^3 field
    assert bench.matched_profile(0.01, light, 16) == ("cosh_4d", 0.2)
    assert bench.matched_profile(0.8, light, 16)[0] == "cosh_t"


def test_light_residue_divides_by_the_profile_range():
    dims = (64, 32, 32, 32)
    prof = ("cosh_4d", 0.2)
    rng = math.cosh(0.2 * 32) * math.cosh(0.2 * 16) ** 3
    assert abs(bench.profile_range(prof, dims) / rng - 1) < 1e-12
    assert bench.light_residue(1e-10, prof, dims) == max(1e-10 / rng, 3e-14)
    assert bench.light_residue(1e-10, ("cosh_t", 0.5), dims) == 1e-10
    assert bench.light_residue(1e-6, prof, (16, 8, 8, 8)) > 3e-14


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
