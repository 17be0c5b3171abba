"""The benchmark's roofline arithmetic for the search kernel, on synthetic
measured peaks (host logic only): the achieved rate is evaluations per
second times the IMAD-equivalents of one evaluation, each multiply form
weighted by its measured cost relative to mad.lo.u32, and the peak is scaled
to the SM clock of the timed region."""
import pytest

import bench


def peaks(imad=19.2e12, wide=7.6e12, hi=8.6e12, mixed=37.0e12, mul64=4.6e12, mhz=2031.0):
    row = lambda v: {"per_s": v, "sm_mhz": mhz}  # noqa: E731
    return {"imad": row(imad), "imad_wide": row(wide), "imad_hi": row(hi),
            "imad+lop3": row(mixed), "mul64": row(mul64)}


def test_forms_are_the_evaluations_multiplies():
    """Two 64 x 64-bit products of the remix (one wide and two plain each)
    and the digit sum's remainder (one high, one plain): 8 multiplies."""
    f = bench.IMAD_FORMS_PER_EVAL
    assert f == {"mad.wide.u32": 2, "mad.lo.u32": 5, "mad.hi.u32": 1}
    assert sum(f.values()) == 8
    assert bench.OPS_PER_EVAL == 26


def test_weighted_fraction():
    p = peaks()
    evals, ms = 6.0e12, 6000.0
    r = bench.search_roofline(p, evals, ms, 2031.0, None)
    w_wide, w_hi = 19.2e12 / 7.6e12, 19.2e12 / 8.6e12
    eq = 2 * w_wide + 5 + w_hi
    assert r["imad_equivalents_per_eval"] == pytest.approx(eq)
    assert r["achieved"] == pytest.approx(evals / 6.0 * eq / 1e12)
    assert r["frac"] == pytest.approx(evals / 6.0 * eq / 19.2e12)
    assert r["frac_unweighted"] == pytest.approx(evals / 6.0 * 8 / 19.2e12)
    assert r["issue"]["frac"] == pytest.approx(evals / 6.0 * 26 / 37.0e12)
    assert r["mul64_check"]["predicted_equiv"] == pytest.approx(w_wide + 2)
    assert r["mul64_check"]["measured_equiv"] == pytest.approx(19.2e12 / 4.6e12)


def test_peak_follows_the_timed_clock():
    """A run at a lower SM clock than the microbenchmark's is held against a
    proportionally lower peak, so the fraction does not change with clocks."""
    p = peaks(mhz=2000.0)
    full = bench.search_roofline(p, 6.0e12, 6000.0, 2000.0, None)
    slow = bench.search_roofline(p, 6.0e12 * 0.9, 6000.0, 1800.0, None)
    assert slow["peak"] == pytest.approx(full["peak"] * 0.9)
    assert slow["frac"] == pytest.approx(full["frac"])
    # no clock sample: the peak is taken as measured
    none = bench.search_roofline(p, 6.0e12, 6000.0, None, None)
    assert none["peak"] == pytest.approx(19.2)


def test_traffic_is_reported_as_given():
    r = bench.search_roofline(peaks(), 6.0e12, 6000.0, 2031.0, 94.0e6)
    assert r["traffic"] == 94.0e6 and r["bound"] == "alu" and r["kernel"] == "k_search"
