"""Materialisation decisions and left-deep join order from exact counts
(host logic of planner.py; no GPU)."""
import itertools

import numpy as np

from paper_1901_01488_gb300.planner import Policy, decide, join_order


def test_policy_thresholds_and_probe():
    rels = [("fact", 1_000_000, True), ("d0", 50_000, True), ("d1", 40_000, True), ("d2", 900, True),
            ("d3", 20_000, False)]
    counts = {"fact": 300_000, "d0": 500, "d1": 30_000}
    d = decide(rels, counts, Policy(min_rows=1_000, max_sel=0.5))
    assert d["fact"].probe and d["fact"].subqueried and not d["fact"].pushed_down   # probe side: never pushed down
    assert d["d0"].pushed_down and d["d0"].cardinality == 500                         # 1 % < 50 %
    assert not d["d1"].pushed_down and d["d1"].cardinality == 30_000                  # 75 % >= 50 %: discarded
    assert not d["d2"].subqueried and d["d2"].cardinality == 900                      # not above min_rows
    assert not d["d3"].subqueried and d["d3"].cardinality == 20_000                   # no selection
    # the selectivity threshold is strict, and min_rows is strict
    d = decide([("f", 10, True), ("a", 4, True)], {"f": 1, "a": 2}, Policy(min_rows=3, max_sel=0.5))
    assert not d["a"].pushed_down
    d = decide([("f", 10, True), ("a", 4, True)], {"f": 1, "a": 1}, Policy(min_rows=4, max_sel=0.5))
    assert not d["a"].subqueried


def test_star_order_is_by_cardinality():
    rels = [("fact", 10**6, False)] + [(f"d{i}", 10**5, True) for i in range(4)]
    counts = {"d0": 70, "d1": 5, "d2": 900, "d3": 5}
    d = decide(rels, counts, Policy())
    order = join_order(d, [("fact", f"d{i}") for i in range(4)])
    assert order == ["fact", "d1", "d3", "d0", "d2"]          # ties by name


def test_chain_waits_for_connectivity():
    # Y is smallest but joins only X: X comes first (no Cartesian product)
    rels = [("F", 1000, False), ("X", 500, False), ("Y", 5, False), ("Z", 50, False)]
    d = decide(rels, {}, Policy())
    assert join_order(d, [("F", "X"), ("X", "Y"), ("F", "Z")]) == ["F", "Z", "X", "Y"]
    # a relation joined to nothing comes last, by a Cartesian product
    assert join_order(d, [("F", "X"), ("X", "Y")]) == ["F", "X", "Y", "Z"]


def test_greedy_definition_on_random_graphs():
    """Brute check of the rule itself: every step picks, among relations that
    share a join predicate with those joined (all others if none does), one
    of least cardinality."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        k = int(rng.integers(2, 7))
        names = [f"r{i}" for i in range(k)]
        sizes = rng.integers(1, 1000, k)
        rels = [(n, int(s), False) for n, s in zip(names, sizes)]
        edges = [e for e in itertools.combinations(names, 2) if rng.random() < 0.4]
        d = decide(rels, {}, Policy())
        order = join_order(d, edges)
        assert sorted(order) == sorted(names)
        assert order[0] == max(names, key=lambda n: (d[n].nrows, n))
        for i in range(1, k):
            joined = set(order[:i])
            adj = {b for a, b in edges if a in joined} | {a for a, b in edges if b in joined}
            cand = (adj - joined) or (set(names) - joined)
            assert order[i] in cand
            assert d[order[i]].cardinality == min(d[n].cardinality for n in cand)
