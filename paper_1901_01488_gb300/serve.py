"""Serving loop for selectivity sub-queries: continuous batching over resident tables.

Not in the paper (there, the optimizer issues one sub-query per table with
a selection, Sec. 2); this is the serving pattern around it.  Requests
(table, predicate) arrive over time.  A host loop keeps `streams` waves in
flight: whenever a stream is free it admits every request that has arrived,
up to `max_batch` and within the device-memory budget (each request reserves
the scratch and output bytes its materialisation needs), compiles their
predicates and launches them: count requests on one table, when at least
`shared_min` of them arrived together, share one pass over it
(esc_selectivity_shared_async); the others run as one batch
(esc_selectivity_batch_async).
Waves on different streams overlap on the GPU.  A request's latency runs
from its arrival to the host observing its wave's completion event.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Deque, Dict, List, Optional, Sequence

import numpy as np
import torch


@dataclasses.dataclass
class Request:
    rid: int
    table: int                 # index into the server's tables
    text: str                  # predicate
    arrival: float             # seconds, on the server's clock
    proj: Sequence[str] = ()   # projection to materialise, () = count only
    capacity: int = 0          # output rows reserved when materialising
    count: Optional[int] = None
    done: Optional[float] = None
    rows: Optional[tuple] = None


def request_bytes(nrows: int, req: Request, widths: Dict[str, int]) -> int:
    """Device memory a request holds while in flight: library scratch for
    materialisation (the selection bitmap, 1/8 byte per row, and 16 bytes
    per work unit of at least 2048 rows) and its output buffers."""
    if not req.proj:
        return 256
    scratch = nrows // 8 + nrows // 128 + 4096
    return scratch + req.capacity * (4 + sum(widths[c] for c in req.proj))


class Server:
    def __init__(self, esc, tables, mem_budget: int = 8 << 30, max_batch: int = 512, streams: int = 2,
                 device="cuda", shared_min: int = 8):
        self.esc = esc
        self.tables = tables
        self.budget = mem_budget
        self.max_batch = max_batch
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.widths = [{n: esc.WIDTH[d] for n, d, _ in t.columns} for t in tables]
        self.in_flight_bytes = 0
        self.peak_bytes = 0
        self.waves = 0
        self.shared_min = shared_min      # count requests per table that share one pass
        self.shared_launches = 0

    def run(self, requests: Sequence[Request], clock=time.perf_counter) -> List[Request]:
        """Serves `requests` (arrival times relative to the start) and returns them completed."""
        esc = self.esc
        pending: Deque[Request] = deque()
        queue = deque(sorted(requests, key=lambda r: r.arrival))
        slots: List[Optional[dict]] = [None] * len(self.streams)
        t0 = clock()
        done_n = 0
        while done_n < len(requests):
            now = clock() - t0
            while queue and queue[0].arrival <= now:
                pending.append(queue.popleft())
            progressed = False
            for k, st in enumerate(self.streams):
                w = slots[k]
                if w is not None and w["event"].query():
                    t_done = clock() - t0
                    counts = w["counts"].tolist()
                    for r, c in zip(w["reqs"], counts):
                        r.count = int(c)
                        r.done = t_done
                    self.in_flight_bytes -= w["bytes"]
                    done_n += len(w["reqs"])
                    slots[k] = None
                    progressed = True
                if slots[k] is None and pending:
                    batch, nbytes = [], 0
                    while pending and len(batch) < self.max_batch:
                        r = pending[0]
                        b = request_bytes(self.tables[r.table].nrows, r, self.widths[r.table])
                        # admission by device memory; a request larger than the
                        # whole budget runs alone once nothing else is in flight
                        alone = not batch and self.in_flight_bytes == 0
                        if self.in_flight_bytes + nbytes + b > self.budget and not alone:
                            break
                        batch.append(pending.popleft())
                        nbytes += b
                    if batch:
                        self._launch(batch, k, st, nbytes, slots)
                        progressed = True
            if not progressed:
                time.sleep(20e-6)
        return list(requests)

    def _launch(self, batch: List[Request], k: int, st, nbytes: int, slots) -> None:
        esc = self.esc
        # count requests on one table, when there are enough of them, share one
        # pass over it; the rest run as one batch.  Shared groups come first.
        per_table: Dict[int, List[Request]] = {}
        for r in batch:
            if not r.proj:
                per_table.setdefault(r.table, []).append(r)
        shared = {ti for ti, rs in per_table.items() if len(rs) >= self.shared_min}
        batch = ([r for r in batch if not r.proj and r.table in shared] +
                 [r for r in batch if r.proj or r.table not in shared])
        preds = []
        rows = []
        for r in batch:
            t = self.tables[r.table]
            p = esc.Predicate(t, r.text, tuple(r.proj))
            preds.append(p)
            if r.proj:
                r.rows = p.alloc_rows(max(1, r.capacity), device=self.device)
                rows.append(r.rows)
            else:
                rows.append(None)
        counts = torch.zeros(len(batch), dtype=torch.int64, device=self.device)
        with torch.cuda.stream(st):
            i = 0
            while i < len(batch) and not batch[i].proj and batch[i].table in shared:
                j = i
                while j < len(batch) and not batch[j].proj and batch[j].table == batch[i].table:
                    j += 1
                esc.esc_selectivity_shared_async(self.tables[batch[i].table].handle, [p.handle for p in preds[i:j]],
                                                 counts[i:j], st)
                self.shared_launches += 1
                i = j
            if i < len(batch):
                rest = rows[i:]
                esc.esc_selectivity_batch_async([self.tables[r.table].handle for r in batch[i:]],
                                                [p.handle for p in preds[i:]], counts[i:],
                                                rest if any(x is not None for x in rest) else None, None, st)
            ev = torch.cuda.Event()
            ev.record(st)
        self.in_flight_bytes += nbytes
        self.peak_bytes = max(self.peak_bytes, self.in_flight_bytes)
        self.waves += 1
        slots[k] = {"reqs": batch, "counts": counts, "event": ev, "bytes": nbytes, "preds": preds}


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def latency_summary(reqs: Sequence[Request]) -> Dict[str, float]:
    lat = np.array([(r.done - r.arrival) * 1e3 for r in reqs])
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "throughput_per_s": len(reqs) / span}
