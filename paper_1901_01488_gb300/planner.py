"""Exact-selectivity planning on top of libesc: the consumer of the counts.

For a query over relations joined along a join graph, each relation with an
optional selection predicate (paper Sec. 2, Sec. 2.1, Sec. 2.2):

1. ESC phase (Sec. 2, Sec. 2.1).  Every relation that has a selection and
   is large enough for the policy gets its selectivity sub-query: the exact
   count.  Smaller relations are not sub-queried.
2. Materialisation decision (Sec. 2.1, Sec. 2.2).  The largest relation is
   the probe side of the hash joins and its selection is never pushed down;
   every other sub-queried relation whose selectivity the policy admits is
   materialised (its qualifying rows with the projection the rest of the plan
   needs) and registered as an esc table, so that later sub-queries and the
   join run on it instead of the base table.  Relations the policy does not
   admit are not materialised at all.
3. Join order (Sec. 2.2).  Left-deep: probe the largest relation, then
   repeatedly join the relation of smallest cardinality that shares a join
   predicate with those already joined (no Cartesian products while a
   connected relation remains).

Two policies.  `Policy` holds the two parameters of Sec. 2.1 (minimum table
size, maximum selectivity) as fixed values, the paper's DBA setting.
`AdaptivePolicy` derives them per relation from measured costs — the adaptive
algorithm the paper leaves to future work (Sec. 2.1, Sec. 4) — by the
trade-off Sec. 2.1 states: materialising costs a call and extra memory
traffic, and pays off through the rows it prunes from every later read of
the relation.  With N rows, C qualifying, w_base the bytes per row a later
read of the base relation touches (predicate and projected columns), w_proj
the bytes per row of the materialised result, u the reads a materialised
result serves, d the seconds per byte of a scan and a + b C the measured cost
of materialising C rows:

    materialise  <=>  u d (N w_base - C w_proj)  >  a + b C
                 <=>  C / N  <  (u d w_base - a / N) / (u d w_proj + b),

so the maximum selectivity grows with N towards u d w_base / (u d w_proj + b),
and below N = a / (u d w_base) nothing is admitted (the minimum size, which
Sec. 2.1 motivates by materialisation: only large tables leave room for the
reduction).  The count itself is cheap and pays through the join order, which
the planner cannot price, so the adaptive policy counts every relation with a
selection above a fixed `count_min_rows` (default 0).  d, a
and b are least-squares fits, with exponential forgetting, of the planner's
own CUDA-event timings of its count calls (scan time against bytes read) and
select calls (select minus count time against rows materialised); u is the
mean number of reads per materialised result: one by the join it was made
for, plus every later plan that uses it as a relation.

Readings where the paper is silent: a relation without a sub-query counts
with its base size (the engine the paper extends keeps no estimates); the
probe side is the largest base relation; ties are broken by name.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional, Sequence, Tuple

import torch

WIDTH = {"u8": 1, "u16": 2, "i32": 4, "i64": 8}


@dataclasses.dataclass
class Relation:
    name: str
    table: object                 # esc.Table
    pred: Optional[str] = None    # selection predicate, or None
    proj: Sequence[str] = ()      # columns the rest of the plan needs


# Bytes per row of a relation: (a later read of the base relation: predicate
# and projected columns, the materialised result: projected columns).
Widths = Tuple[int, int]


@dataclasses.dataclass
class Policy:
    """The two parameters of Sec. 2.1, fixed (the DBA's setting)."""
    min_rows: int = 0             # ESC only for relations with more rows
    max_sel: float = 1.0          # materialise only below this selectivity

    def min_rows_for(self, widths: Widths) -> float:
        return self.min_rows

    def max_sel_for(self, nrows: int, widths: Widths) -> float:
        return self.max_sel

    def subquery(self, nrows: int, widths: Widths) -> bool:
        return nrows > self.min_rows

    def admits(self, nrows: int, count: int, widths: Widths) -> bool:
        sel = count / nrows if nrows else 1.0
        return sel < self.max_sel_for(nrows, widths)


class LineFit:
    """Weighted least squares of t = a + b x with exponential forgetting: each
    observation multiplies the weight of all earlier ones by `forget`.  A prior
    line enters as two pseudo-observations (x = 0 and x = x_ref) of weight
    `prior_weight` each, so the fit is defined before any observation and the
    prior fades as observations arrive.  a and b are kept non-negative."""

    def __init__(self, a0: float, b0: float, x_ref: float, prior_weight: float = 1.0, forget: float = 0.95):
        self.forget = forget
        self.s = [0.0] * 5                     # sums of w, w x, w t, w x^2, w x t
        self.n = 0
        for x in (0.0, x_ref):
            self._add(x, a0 + b0 * x, prior_weight)

    def _add(self, x: float, t: float, w: float):
        s = self.s
        s[0] += w
        s[1] += w * x
        s[2] += w * t
        s[3] += w * x * x
        s[4] += w * x * t

    def observe(self, x: float, t: float):
        self.s = [v * self.forget for v in self.s]
        self._add(float(x), float(t), 1.0)
        self.n += 1

    def params(self) -> Tuple[float, float]:
        w, sx, st, sxx, sxt = self.s
        mx, mt = sx / w, st / w
        vxx = sxx / w - mx * mx                # weighted variance of x (the prior keeps it > 0)
        b = (sxt / w - mx * mt) / vxx if vxx > 0 else 0.0
        b = max(b, 0.0)
        a = mt - b * mx
        if a < 0.0:                            # through the origin
            a, b = 0.0, (sxt / sxx if sxx > 0 else 0.0)
        return a, max(b, 0.0)


class AdaptivePolicy(Policy):
    """Minimum size and maximum selectivity per relation from measured costs
    (the cost/benefit rule in the module docstring).

    Units inside: scan x in GB, materialisation x in millions of rows, t in
    seconds.  The priors (scans at 5 TB/s plus 10 us per call, materialising
    at 30 us per call plus 8 ps per row, one read per result) only set the
    first decisions; observations replace them."""

    def __init__(self, scan_gbs: float = 5000.0, scan_fixed_s: float = 10e-6, mat_fixed_s: float = 30e-6,
                 mat_per_row_s: float = 8e-12, uses: float = 1.0, prior_weight: float = 1.0, forget: float = 0.95,
                 count_min_rows: int = 0):
        super().__init__()
        self.count_min_rows = count_min_rows
        self.scan = LineFit(scan_fixed_s, 1.0 / scan_gbs, 1.0, prior_weight, forget)            # t(GB)
        self.mat = LineFit(mat_fixed_s, mat_per_row_s * 1e6, 10.0, prior_weight, forget)         # t(M rows)
        self.use_prior = (uses, 1.0)           # (value, weight)
        self.results = 0                       # materialised results seen
        self.reads = 0                         # reads they served

    # ---------------------------------------------------------------- observations
    def observe_scan(self, nbytes: float, seconds: float):
        self.scan.observe(nbytes / 1e9, seconds)

    def observe_materialise(self, rows: float, seconds: float):
        self.mat.observe(rows / 1e6, max(seconds, 0.0))

    def observe_result(self):
        """A result was materialised: it serves its own join (one read)."""
        self.results += 1
        self.reads += 1

    def observe_reuse(self):
        """A later plan read a materialised result."""
        self.reads += 1

    # ---------------------------------------------------------------- model
    def uses(self) -> float:
        u0, w0 = self.use_prior
        return (u0 * w0 + self.reads) / (w0 + self.results)

    def params(self) -> Dict[str, float]:
        """d (s/byte), a (s), b (s/row), u."""
        _, d_gb = self.scan.params()
        a, b_m = self.mat.params()
        return {"d": d_gb / 1e9, "a": a, "b": b_m / 1e6, "u": self.uses()}

    def min_rows_for(self, widths: Widths) -> float:
        """Minimum size for materialising (an empty result pays from here)."""
        p = self.params()
        gain = p["u"] * p["d"] * widths[0]
        return p["a"] / gain if gain > 0 else float("inf")

    def subquery(self, nrows: int, widths: Widths) -> bool:
        return nrows > self.count_min_rows

    def max_sel_for(self, nrows: int, widths: Widths) -> float:
        p = self.params()
        w_base, w_proj = widths
        if nrows <= 0:
            return 0.0
        num = p["u"] * p["d"] * w_base - p["a"] / nrows
        den = p["u"] * p["d"] * w_proj + p["b"]
        return num / den if den > 0 else (float("inf") if num > 0 else 0.0)

    def admits(self, nrows: int, count: int, widths: Widths) -> bool:
        p = self.params()
        w_base, w_proj = widths
        benefit = p["u"] * p["d"] * (nrows * w_base - count * w_proj)
        return benefit > p["a"] + p["b"] * count


@dataclasses.dataclass
class Decision:
    name: str
    nrows: int
    subqueried: bool
    count: Optional[int]          # exact count when sub-queried
    probe: bool
    pushed_down: bool             # materialised result kept as a temporary table
    cardinality: int              # what the join order uses
    min_rows: float = 0.0         # the policy's thresholds for this relation when decided: minimum
    max_sel: float = 1.0          # size (to sub-query, or for AdaptivePolicy to materialise), maximum selectivity


@dataclasses.dataclass
class Plan:
    decisions: Dict[str, Decision]
    order: List[str]              # left-deep: order[0] is probed, then the builds in join order
    esc_seconds: float            # wall time of the ESC phase (sub-queries + materialisation)
    temp: Dict[str, object]       # name -> esc.Table over the materialised columns


def decide(rels: Sequence[Tuple[str, int, bool]], counts: Dict[str, int], policy: Policy,
           widths: Optional[Dict[str, Widths]] = None,
           materialisable: Optional[set] = None) -> Dict[str, Decision]:
    """Materialisation decisions from (name, base rows, has selection), the
    exact counts of the sub-queried relations, (for a cost-based policy) each
    relation's widths, and the relations that have a projection to
    materialise (None: all)."""
    widths = widths or {}
    probe = max(rels, key=lambda r: (r[1], r[0]))[0]
    out = {}
    for name, nrows, has_sel in rels:
        w = widths.get(name, (0, 0))
        sub = has_sel and policy.subquery(nrows, w)
        cnt = counts.get(name) if sub else None
        push = (sub and name != probe and (materialisable is None or name in materialisable)
                and policy.admits(nrows, cnt, w))
        card = cnt if sub else nrows
        out[name] = Decision(name, nrows, sub, cnt, name == probe, push, card,
                             policy.min_rows_for(w), policy.max_sel_for(nrows, w))
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


def read_widths(pred, table, proj: Sequence[str]) -> Tuple[int, Widths]:
    """(bytes per row the predicate reads, (w_base, w_proj)) of a compiled
    predicate, from the library's program listing."""
    refs = []
    for line in pred.explain().splitlines():
        f = line.split()
        if f and f[0] == "ref":
            refs.append((f[2], f[3]))
    w_pred = sum(WIDTH[t] for _, t in refs)
    names = {n for n, _ in refs}
    w_proj = sum(WIDTH[table.dtype(c)] for c in proj)
    w_base = w_pred + sum(WIDTH[table.dtype(c)] for c in proj if c not in names)
    return w_pred, (w_base, w_proj)


class Planner:
    """Runs the ESC phase through libesc and plans the joins.  With an
    AdaptivePolicy it also feeds the policy its measurements: every count call
    (scan time against bytes read), every materialisation (select minus count
    time against rows) and every later read of a materialised result."""

    def __init__(self, esc, policy: Policy = Policy(), device="cuda"):
        self.esc = esc
        self.policy = policy
        self.device = torch.device(device)
        self._keep: List[object] = []
        self._temps: Dict[int, str] = {}      # id of a registered temporary table -> its relation

    def _events(self, on: bool):
        if not on:
            return None
        st = torch.cuda.current_stream(self.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        return e0, e1, st

    @staticmethod
    def _seconds(ev) -> float:
        return ev[0].elapsed_time(ev[1]) / 1e3

    def plan(self, relations: Sequence[Relation], edges: Sequence[Tuple[str, str]]) -> Plan:
        esc = self.esc
        adaptive = isinstance(self.policy, AdaptivePolicy)
        rels = {r.name: r for r in relations}
        meta = [(r.name, r.table.nrows, r.pred is not None) for r in relations]
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        preds, widths, counts, ev_count, w_read = {}, {}, {}, {}, {}
        for r in relations:
            if adaptive and id(r.table) in self._temps:
                self.policy.observe_reuse()
            if r.pred is None:
                continue
            if not self.policy.subquery(r.table.nrows, (0, 0)):
                continue
            p = esc.Predicate(r.table, r.pred, tuple(r.proj))
            if adaptive:                                  # the fixed policy prices nothing
                w_read[r.name], widths[r.name] = read_widths(p, r.table, r.proj)
            preds[r.name] = p
            ev = self._events(adaptive)
            counts[r.name] = esc.count(r.table, p)       # synchronises: the event below is already due
            if ev:
                ev[1].record(ev[2])
                ev_count[r.name] = ev
        if ev_count:
            torch.cuda.synchronize(self.device)
            for name, ev in ev_count.items():
                self.policy.observe_scan(rels[name].table.nrows * w_read[name], self._seconds(ev))
        decisions = decide(meta, counts, self.policy, widths, {r.name for r in relations if r.proj})
        temp, ev_sel = {}, {}
        for name, dec in decisions.items():
            if not dec.pushed_down:
                continue
            r, p = rels[name], preds[name]
            out = p.alloc_rows(max(1, dec.count), device=self.device)
            ev = self._events(adaptive)
            got, _ = esc.esc_selectivity(r.table.handle, p.handle, out)
            if ev:
                ev[1].record(ev[2])
                ev_sel[name] = ev
            assert got == dec.count, (name, got, dec.count)
            temp[name] = self.register_temp(r, out, dec.count)
        torch.cuda.synchronize(self.device)
        for name, ev in ev_sel.items():
            self.policy.observe_materialise(decisions[name].count, self._seconds(ev) - self._seconds(ev_count[name]))
            self.policy.observe_result()
        esc_s = time.perf_counter() - t0
        return Plan(decisions, join_order(decisions, edges), esc_s, temp)

    def register_temp(self, rel: Relation, out, count: int):
        """A materialised result as an esc table of its projected columns."""
        esc = self.esc
        _, ids, cols = out
        kinds = {n: d for n, d, _ in rel.table.columns}
        columns = [(name, kinds[name], col[:count]) for name, col in zip(rel.proj, cols)]
        self._keep.append((ids, cols))
        t = esc.Table(columns, count)
        self._temps[id(t)] = rel.name
        self._keep.append(t)
        return t

    def drop_temps(self):
        """Releases every temporary table this planner registered."""
        self._keep.clear()
        self._temps.clear()
