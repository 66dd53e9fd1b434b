"""The planner end to end on a star schema: exact counts, materialised
temporary tables and their reuse, checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def esc():
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc as m
    return m


def test_star_plan_and_temp_table_reuse(esc):
    from paper_1901_01488_gb300.planner import Planner, Policy, Relation
    fact = datagen.star_fact(3_000_017, seed=4, device="cuda")
    dims = [datagen.star_dim(d, n, seed=4, device="cuda") for d, n in enumerate(datagen.STAR_DIM_ROWS)]
    texts = datagen.star_dim_predicates(4)
    rels = [Relation("fact", esc.Table.from_datagen(fact), "m0 < 50000", ("fk0", "fk1"))]
    for d, (dim, text) in enumerate(zip(dims, texts)):
        rels.append(Relation(f"dim{d}", esc.Table.from_datagen(dim), text, ("a", "c")))
    policy = Policy(min_rows=10_000, max_sel=0.2)
    plan = Planner(esc, policy).plan(rels, [("fact", f"dim{d}") for d in range(4)])
    host = {r.name: h for r, h in zip(rels, [fact.host()] + [d.host() for d in dims])}
    card = {}
    for r in rels:
        dec = plan.decisions[r.name]
        if dec.subqueried:
            assert dec.count == oracle.count(r.pred, host[r.name]), r.name
        card[r.name] = dec.cardinality
        sel = dec.count / r.table.nrows if dec.subqueried else 1.0
        assert dec.pushed_down == (dec.subqueried and not dec.probe and sel < policy.max_sel)
    assert plan.decisions["fact"].probe and not plan.decisions["fact"].pushed_down
    assert not plan.decisions["dim3"].subqueried            # 2,556 rows: below min_rows
    assert plan.order[0] == "fact"
    assert plan.order[1:] == sorted(plan.order[1:], key=lambda n: (card[n], n))
    assert plan.temp, "at least one dimension is selective enough to be kept"
    for name, tmp in plan.temp.items():
        r = next(x for x in rels if x.name == name)
        ids, vals = oracle.select(r.pred, host[name], list(r.proj))
        assert tmp.nrows == len(ids)
        for (cname, _, t) in tmp.columns:
            assert np.array_equal(t.cpu().numpy().astype(np.int64), vals[cname].astype(np.int64)), (name, cname)
        # a later sub-query on the temporary table = the conjunction on the base table
        follow = "c < 12"
        p = esc.Predicate(tmp, follow)
        assert esc.count(tmp, p) == oracle.count(f"({r.pred}) AND {follow}", host[name])


def test_adaptive_policy_on_the_star_schema(esc):
    """The adaptive policy end to end: its measurements (one scan per
    sub-query, one materialisation per kept result, one reuse per later plan
    that reads a kept result), decisions consistent with the thresholds it
    reported, and exact counts and materialised rows.  The policy's prior
    says each result is read 50 times, so that the 2M-row dimension pays for
    materialising at GB300 scan speed (with one read it would not)."""
    from paper_1901_01488_gb300.planner import AdaptivePolicy, Planner, Relation
    fact = datagen.star_fact(3_000_017, seed=5, device="cuda")
    dims = [datagen.star_dim(d, n, seed=5, device="cuda") for d, n in enumerate(datagen.STAR_DIM_ROWS)]
    texts = datagen.star_dim_predicates(5)
    rels = [Relation("fact", esc.Table.from_datagen(fact), "m0 < 50000", ("fk0", "fk1"))]
    for d, (dim, text) in enumerate(zip(dims, texts)):
        rels.append(Relation(f"dim{d}", esc.Table.from_datagen(dim), text, ("a", "c")))
    host = {r.name: h for r, h in zip(rels, [fact.host()] + [d.host() for d in dims])}
    pol = AdaptivePolicy(uses=50.0)
    planner = Planner(esc, pol)
    edges = [("fact", f"dim{d}") for d in range(4)]
    plan = planner.plan(rels, edges)
    sub = [d for d in plan.decisions.values() if d.subqueried]
    pushed = [d for d in plan.decisions.values() if d.pushed_down]
    assert pol.scan.n == len(sub) and pol.mat.n == len(pushed) and pol.results == len(pushed)
    assert "dim0" in {d.name for d in pushed}, "the 2M-row dimension is worth materialising with 50 reads"
    for d in plan.decisions.values():
        assert d.subqueried                     # every relation with a selection is counted
        assert not d.pushed_down or d.nrows > d.min_rows
        if d.subqueried:
            assert d.count == oracle.count(next(r.pred for r in rels if r.name == d.name), host[d.name])
            margin = abs(d.count - d.max_sel * d.nrows)
            if not d.probe and margin > 1e-6 * d.nrows:
                assert d.pushed_down == (d.count < d.max_sel * d.nrows), d
        if d.probe:
            assert not d.pushed_down
    assert set(plan.temp) == {d.name for d in pushed}
    for name, tmp in plan.temp.items():
        r = next(x for x in rels if x.name == name)
        ids, vals = oracle.select(r.pred, host[name], list(r.proj))
        assert tmp.nrows == len(ids)
        for (cname, _, t) in tmp.columns:
            assert np.array_equal(t.cpu().numpy().astype(np.int64), vals[cname].astype(np.int64)), (name, cname)
    # a later plan reading a kept result counts as a reuse
    reads = pol.reads
    name, tmp = next(iter(plan.temp.items()))
    follow = planner.plan([Relation("fact", rels[0].table, "m0 < 50000", ("fk0",)),
                           Relation(name + "_kept", tmp, "c < 12", ("a",))], [("fact", name + "_kept")])
    assert pol.reads == reads + 1
    r = next(x for x in rels if x.name == name)
    assert follow.decisions[name + "_kept"].count == oracle.count(f"({r.pred}) AND c < 12", host[name])
    planner.drop_temps()
