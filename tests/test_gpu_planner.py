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
