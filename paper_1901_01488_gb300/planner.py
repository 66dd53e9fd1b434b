"""Exact-selectivity planning on top of libesc: the consumer of the counts.

For a query over relations joined along a join graph, each relation with an
optional selection predicate (paper Sec. 2, Sec. 2.1, Sec. 2.2):

1. ESC phase (Sec. 2, Sec. 2.1).  Every relation that has a selection and
   more rows than `min_rows` gets its selectivity sub-query: the exact count,
   with the projection the rest of the plan needs pushed down and the
   qualifying rows materialised.  Smaller relations are not sub-queried.
2. Materialisation decision (Sec. 2.1, Sec. 2.2).  The largest relation is
   the probe side of the hash joins and its selection is never pushed down;
   every other relation keeps its materialised result as a temporary table
   when its selectivity is below `max_sel`, otherwise the result is
   discarded.  A kept result is registered as an esc table (its projected
   columns), so that later sub-queries run on it instead of the base table.
3. Join order (Sec. 2.2).  Left-deep: probe the largest relation, then
   repeatedly join the relation of smallest cardinality that shares a join
   predicate with those already joined (no Cartesian products while a
   connected relation remains).

Readings where the paper is silent: a relation without a sub-query counts
with its base size (the engine the paper extends keeps no estimates); the
probe side is the largest base relation; ties are broken by name.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import torch


@dataclasses.dataclass
class Relation:
    name: str
    table: object                 # esc.Table
    pred: Optional[str] = None    # selection predicate, or None
    proj: Sequence[str] = ()      # columns the rest of the plan needs


@dataclasses.dataclass
class Policy:
    min_rows: int = 0             # ESC only for relations with more rows
    max_sel: float = 1.0          # materialise only below this selectivity


@dataclasses.dataclass
class Decision:
    name: str
    nrows: int
    subqueried: bool
    count: Optional[int]          # exact count when sub-queried
    probe: bool
    pushed_down: bool             # materialised result kept as a temporary table
    cardinality: int              # what the join order uses


@dataclasses.dataclass
class Plan:
    decisions: Dict[str, Decision]
    order: List[str]              # left-deep: order[0] is probed, then the builds in join order
    esc_seconds: float            # wall time of the ESC phase (sub-queries + materialisation)
    temp: Dict[str, object]       # name -> esc.Table over the materialised columns


def decide(rels: Sequence[Tuple[str, int, bool]], counts: Dict[str, int], policy: Policy) -> Dict[str, Decision]:
    """Materialisation decisions from (name, base rows, has selection) and the
    exact counts of the sub-queried relations."""
    probe = max(rels, key=lambda r: (r[1], r[0]))[0]
    out = {}
    for name, nrows, has_sel in rels:
        sub = has_sel and nrows > policy.min_rows
        cnt = counts.get(name) if sub else None
        sel = (cnt / nrows) if (sub and nrows) else 1.0
        push = sub and name != probe and sel < policy.max_sel
        card = cnt if sub else nrows
        out[name] = Decision(name, nrows, sub, cnt, name == probe, push, card)
    return out


def join_order(decisions: Dict[str, Decision], edges: Sequence[Tuple[str, str]]) -> List[str]:
    """Left-deep order: the probe first, then greedily the smallest connected relation."""
    adj: Dict[str, set] = {n: set() for n in decisions}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    probe = next(n for n, d in decisions.items() if d.probe)
    order, joined = [probe], {probe}
    while len(order) < len(decisions):
        frontier = {n for j in joined for n in adj[j]} - joined
        pool = frontier if frontier else set(decisions) - joined   # a Cartesian product only if unavoidable
        nxt = min(pool, key=lambda n: (decisions[n].cardinality, n))
        order.append(nxt)
        joined.add(nxt)
    return order


class Planner:
    """Runs the ESC phase through libesc and plans the joins."""

    def __init__(self, esc, policy: Policy = Policy(), device="cuda"):
        self.esc = esc
        self.policy = policy
        self.device = torch.device(device)
        self._keep: List[object] = []

    def plan(self, relations: Sequence[Relation], edges: Sequence[Tuple[str, str]]) -> Plan:
        esc = self.esc
        rels = {r.name: r for r in relations}
        meta = [(r.name, r.table.nrows, r.pred is not None) for r in relations]
        probe = max(meta, key=lambda m: (m[1], m[0]))[0]
        counts: Dict[str, int] = {}
        rows: Dict[str, tuple] = {}
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        for name, nrows, has_sel in meta:
            if not (has_sel and nrows > self.policy.min_rows):
                continue
            r = rels[name]
            p = esc.Predicate(r.table, r.pred, tuple(r.proj))
            if name == probe or not r.proj:
                counts[name] = esc.count(r.table, p)      # never pushed down: the count alone
            else:
                n = esc.count(r.table, p)
                out = p.alloc_rows(max(1, n), device=self.device)
                got, _ = esc.esc_selectivity(r.table.handle, p.handle, out)
                counts[name] = got
                rows[name] = (p, out)
        decisions = decide(meta, counts, self.policy)
        temp = {}
        for name, (p, out) in rows.items():
            if decisions[name].pushed_down:
                temp[name] = self.register_temp(rels[name], out, decisions[name].count)
        torch.cuda.synchronize(self.device)
        esc_s = time.perf_counter() - t0
        return Plan(decisions, join_order(decisions, edges), esc_s, temp)

    def register_temp(self, rel: Relation, out, count: int):
        """A materialised result as an esc table of its projected columns."""
        esc = self.esc
        _, ids, cols = out
        kinds = {n: d for n, d, _ in rel.table.columns}
        columns = [(name, kinds[name], col[:count]) for name, col in zip(rel.proj, cols)]
        self._keep.append((ids, cols))
        return esc.Table(columns, count)
