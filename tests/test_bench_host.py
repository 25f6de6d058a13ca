"""Host-side pieces of bench.py that need no GPU: the clock/throttle summary and the flop models."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(HERE, "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_reports_median_max_and_active_reasons(bench):
    cs = bench.ClockSampler()
    # rows as nvidia-smi prints them with --format=csv,noheader,nounits, split on commas
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1965, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    cs.samples = [[x.strip() for x in r.split(",")] for r in rows]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0  # the unparsable sample is skipped
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    cs.samples.append([x.strip() for x in "0, 1500, 2070, 700, 0x8, Active, Not Active, Active, Not Active".split(",")])
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples(bench):
    s = bench.ClockSampler().summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_triples_flops_are_a_third_of_the_work_model(bench):
    """The kernels form each sorted virtual triple once: 2o^3v^4 + 2o^4v^3, a third of the
    6o^3v^4 + 6o^4v^3 model that counts the j<->k-symmetric loop over all triples."""
    for o, v in ((4, 24), (16, 240), (32, 480)):
        _, trip = bench.model_flops(o, v, 1)
        assert trip == 3 * bench.triples_algorithmic_flops(o, v)


def test_sorted_triple_count_matches_the_flop_model(bench):
    """Each sorted triple a<=b<=c costs six terms of 2o^3 v (d-part) + 2o^4 (l-part) flops, i.e.
    (2o^3v + 2o^4) * v(v+1)(v+2): the model's 2o^3v^4 + 2o^4v^3 up to the (v+1)(v+2)/v^2 factor."""
    o = 5
    for v in (7, 30):
        brute = sum(6 * (2 * o**3 * v + 2 * o**4) for a in range(v) for b in range(a, v) for c in range(b, v))
        assert brute == (2 * o**3 * v + 2 * o**4) * v * (v + 1) * (v + 2)
        ratio = brute / bench.triples_algorithmic_flops(o, v)
        assert ratio == pytest.approx((v + 1) * (v + 2) / v**2, rel=1e-12)


def test_ccsd_work_model_per_iteration(bench):
    o, v = 16, 240
    c1, _ = bench.model_flops(o, v, 1)
    c9, _ = bench.model_flops(o, v, 9)
    assert c9 == 9 * c1 == 9 * (2 * o**2 * v**4 + 16 * o**3 * v**3 + 2 * o**4 * v**2)
