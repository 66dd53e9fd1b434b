"""Adaptive materialisation thresholds (planner.AdaptivePolicy, LineFit):
host logic, no GPU.

The pins: the fitted lines against exact lines and against a regime change;
the admission rule against a brute-force comparison of the two alternatives'
total times (materialise the result and read it u times, or read the base
relation u times), found by bisection over the count; the minimum size
against the smallest table where an empty result is admitted; learning from
noisy simulated timings against the hidden costs."""
import math
import random

import pytest

from paper_1901_01488_gb300.planner import AdaptivePolicy, LineFit, Policy, decide


def exact_policy(d, a, b, u=1.0):
    """A policy whose fitted parameters are exactly (d, a, b, u): the prior
    lines with no observation (two points on each line) and prior uses u."""
    return AdaptivePolicy(scan_gbs=1.0 / (d * 1e9), scan_fixed_s=0.0, mat_fixed_s=a, mat_per_row_s=b, uses=u)


def test_linefit_recovers_a_line():
    f = LineFit(1.0, 1.0, 1.0, prior_weight=1e-12, forget=1.0)
    for x in (0.5, 1.0, 4.0, 7.0, 7.0):
        f.observe(x, 3.0 + 2.0 * x)
    a, b = f.params()
    assert a == pytest.approx(3.0, rel=1e-9) and b == pytest.approx(2.0, rel=1e-9)


def test_linefit_prior_alone_and_forgetting():
    a, b = LineFit(0.25, 4.0, 10.0).params()
    assert (a, b) == (pytest.approx(0.25), pytest.approx(4.0))
    f = LineFit(0.25, 4.0, 10.0, forget=0.8)
    rng = random.Random(1)
    for _ in range(40):
        x = rng.uniform(0, 10)
        f.observe(x, 1.0 + 1.0 * x)
    for _ in range(80):                      # a new regime: the old one fades (0.8^80 ~ 2e-8)
        x = rng.uniform(0, 10)
        f.observe(x, 5.0 + 0.5 * x)
    a, b = f.params()
    assert a == pytest.approx(5.0, rel=1e-4) and b == pytest.approx(0.5, rel=1e-4)


def test_linefit_keeps_parameters_non_negative():
    f = LineFit(1.0, 1.0, 1.0, prior_weight=1e-12, forget=1.0)
    for x in (1.0, 2.0, 3.0):
        f.observe(x, 10.0 - x)               # negative slope
    assert f.params()[1] == 0.0
    g = LineFit(1.0, 1.0, 1.0, prior_weight=1e-12, forget=1.0)
    for x in (1.0, 2.0, 3.0):
        g.observe(x, -1.0 + 2.0 * x)         # negative intercept: through the origin
    a, b = g.params()
    assert a == 0.0 and b > 0.0


def _total_time(materialise, n, c, d, a, b, u, w_base, w_proj):
    """Time of the two alternatives for a result of c of n rows read u times."""
    if materialise:
        return a + b * c + u * d * c * w_proj
    return u * d * n * w_base


def test_admission_is_the_break_even_of_the_two_alternatives():
    rng = random.Random(7)
    for _ in range(300):
        d = 10 ** rng.uniform(-13, -11)      # 1 .. 100 TB/s
        a = 10 ** rng.uniform(-6, -3)
        b = 10 ** rng.uniform(-13, -9)
        u = rng.uniform(0.5, 6.0)
        w_proj = rng.choice([4, 8, 12, 16, 20])
        w_base = w_proj + rng.choice([0, 1, 2, 4, 8, 13])
        n = rng.randrange(1, 2_000_000_000)
        pol = exact_policy(d, a, b, u)
        # largest count for which materialising is strictly faster (-1: none), by bisection
        lo, hi = -1, n + 1
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if _total_time(True, n, mid, d, a, b, u, w_base, w_proj) < _total_time(False, n, mid, d, a, b, u, w_base, w_proj):
                lo = mid
            else:
                hi = mid
        widths = (w_base, w_proj)
        for c in (lo - 1, lo, lo + 1, lo + 2, 0, n):
            if 0 <= c <= n:
                want = _total_time(True, n, c, d, a, b, u, w_base, w_proj) < _total_time(False, n, c, d, a, b, u, w_base, w_proj)
                assert pol.admits(n, c, widths) == want, (n, c, lo)
        # the threshold: max_sel * n is the break-even count (within a row)
        s = pol.max_sel_for(n, widths)
        if lo >= 0 and s * n <= n:
            assert abs(s * n - (lo + 1)) <= 1.0 + 1e-9 * n, (s * n, lo)
        else:
            assert s <= 0.0 or s * n > n


def test_minimum_size_is_where_an_empty_result_starts_to_pay():
    rng = random.Random(3)
    for _ in range(100):
        d, a, b = 10 ** rng.uniform(-13, -11), 10 ** rng.uniform(-6, -3), 10 ** rng.uniform(-13, -9)
        u = rng.uniform(0.5, 4.0)
        widths = (rng.choice([4, 9, 16, 25]), 4)
        pol = exact_policy(d, a, b, u)
        lo, hi = 0, 1 << 50                  # smallest n with admits(n, 0)
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if pol.admits(mid, 0, widths):
                hi = mid
            else:
                lo = mid
        m = pol.min_rows_for(widths)
        assert abs(m - lo) <= 1.0 + 1e-9 * m, (m, lo)
        assert not pol.admits(int(math.floor(m)), 0, widths) and pol.admits(int(math.floor(m)) + 2, 0, widths)
    # counting is not gated by the learned size
    pol = exact_policy(1e-12, 1e-3, 1e-12)
    assert pol.subquery(1, (4, 4)) and not AdaptivePolicy(count_min_rows=100).subquery(100, (4, 4))


def test_more_reads_raise_the_threshold_and_lower_the_minimum():
    pol = exact_policy(2e-13, 40e-6, 6e-12, u=1.0)
    widths = (13, 16)
    s1, m1 = pol.max_sel_for(60_000_000, widths), pol.min_rows_for(widths)
    pol.observe_result()
    for _ in range(5):
        pol.observe_reuse()
    assert pol.uses() == pytest.approx((1 + 6) / 2)
    assert pol.max_sel_for(60_000_000, widths) > s1 and pol.min_rows_for(widths) < m1
    # a result nobody reads again: uses -> 1
    pol2 = exact_policy(2e-13, 40e-6, 6e-12, u=1.0)
    for _ in range(100):
        pol2.observe_result()
    assert pol2.uses() == pytest.approx(1.0)


def test_learning_from_noisy_timings():
    """Observations made as the planner makes them, from hidden costs with 2 %
    noise: the fits, and the thresholds, come within a few percent."""
    d, e, a, b = 1.0 / 6.5e12, 4e-6, 25e-6, 7e-12
    pol = AdaptivePolicy(forget=0.99)        # priors off by 30-40 %
    rng = random.Random(11)
    for _ in range(400):
        n = rng.choice([2_556, 30_000, 200_000, 2_000_000, 60_000_000, 600_000_000])
        nbytes = n * rng.choice([1, 4, 5, 8, 13, 16, 32])
        pol.observe_scan(nbytes, (e + d * nbytes) * rng.uniform(0.98, 1.02))
        c = int(n * 10 ** rng.uniform(-4, 0))
        pol.observe_materialise(c, (a + b * c) * rng.uniform(0.98, 1.02))
    p = pol.params()
    assert p["d"] == pytest.approx(d, rel=0.03)
    assert p["b"] == pytest.approx(b, rel=0.03)
    assert p["a"] == pytest.approx(a, rel=0.25)          # small against the larger calls' noise
    truth = exact_policy(d, a, b)
    for widths in ((13, 16), (5, 8)):
        assert pol.max_sel_for(60_000_000, widths) == pytest.approx(truth.max_sel_for(60_000_000, widths), rel=0.05)


def test_decide_uses_each_relations_widths():
    pol = exact_policy(1 / 6e12, 30e-6, 8e-12)
    # at 6 TB/s and 30 us per materialisation, a relation read at 40 B/row pays
    # off from 4.5M rows on (an empty result): take 20M-row relations
    rels = [("fact", 600_000_000, True), ("wide", 20_000_000, True), ("narrow", 20_000_000, True),
            ("noproj", 20_000_000, True), ("tiny", 1_000, True)]
    counts = {"fact": 1_000, "wide": 6_000_000, "narrow": 6_000_000, "noproj": 10, "tiny": 1}
    widths = {"fact": (16, 16), "wide": (40, 4), "narrow": (5, 4), "noproj": (40, 0), "tiny": (40, 4)}
    dec = decide(rels, counts, pol, widths, materialisable={"fact", "wide", "narrow", "tiny"})
    assert dec["fact"].probe and not dec["fact"].pushed_down            # the probe side: never
    assert dec["wide"].pushed_down and not dec["narrow"].pushed_down     # same selectivity, different widths
    assert dec["wide"].max_sel > 0.3 > dec["narrow"].max_sel
    assert not dec["noproj"].pushed_down                                 # nothing to materialise
    assert dec["tiny"].subqueried and not dec["tiny"].pushed_down        # counted; below the learned minimum size
    assert dec["tiny"].min_rows > 1_000
    # the fixed policy through the same function: unchanged behaviour
    dec = decide(rels, counts, Policy(min_rows=10_000, max_sel=0.5), widths)
    assert dec["wide"].pushed_down and dec["narrow"].pushed_down and not dec["tiny"].subqueried
