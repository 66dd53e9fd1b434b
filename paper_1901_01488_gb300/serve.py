"""Serving loop for selectivity sub-queries: continuous batching over resident tables.

Not in the paper (there, the optimizer issues one sub-query per table with
a selection, Sec. 2); this is the serving pattern around it.  Requests
(table, predicate) arrive over time.  A host loop keeps `streams` waves in
flight: whenever a stream is free it admits every request that has arrived,
up to `max_batch`, within the device-memory budget (each request reserves the scratch and output bytes
its materialisation needs) and within `max_wave_rows` table rows scanned (a
wave's requests complete together, so one long wave would hold back every
short request in it), and launches them: count requests on one table, when
at least `shared_min` of them arrived together, share one pass over it
(esc_selectivity_shared_async); the others run as one batch
(esc_selectivity_batch_async), or as a plain call when only one is left.
Waves on different streams overlap on the GPU.  A request's predicate is
compiled when it arrives, on the polling thread by default (about 8 us);
`compile_threads` > 0 hands compilation to a pool of host threads instead,
which measured slower: each request then waits for a thread hand-off.  A
request's latency runs from its arrival to the host observing its wave's
completion event.

`PlainServer` is the baseline without batching: every request is its own
sub-query call, launched when it arrives (round robin over the streams).
"""
from __future__ import annotations

import contextlib
import dataclasses
import gc
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from typing import Callable, Deque, Dict, List, Optional, Sequence, Tuple

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
    pred: Optional[object] = None       # compiled predicate (a future while compiling)


class _Ready:
    """A predicate compiled on the polling thread, in the shape of a finished
    future (compile_threads = 0)."""
    __slots__ = ("value",)

    def __init__(self, value):
        self.value = value

    def result(self):
        return self.value

    def done(self) -> bool:
        return True


def _compile_pool(threads: int) -> Optional[ThreadPoolExecutor]:
    return ThreadPoolExecutor(threads) if threads > 0 else None


def request_bytes(nrows: int, req: Request, widths: Dict[str, int]) -> int:
    """Device memory a request holds while in flight: its compiled query and
    counters in the launch (4 KB), and when it materialises, the library's
    scratch (the selection bitmap, 1/8 byte per row rounded up to whole tiles
    of at most 32768 rows; 16 bytes per compaction unit, of which there are
    at most one per 256-row group and at most one per 65536 rows plus one
    wave of write-kernel blocks, taken as 1024; headers) and its output
    buffers."""
    base = 4096
    if not req.proj:
        return base
    units = min((nrows + 255) // 256, (nrows + 65535) // 65536 + 1024)
    scratch = nrows // 8 + 16 * units + 8192
    return base + scratch + req.capacity * (4 + sum(widths[c] for c in req.proj))


def admit(pending: Deque[Request], in_flight: int, budget: int, max_batch: int,
          size: Callable[[Request], int], work: Optional[Callable[[Request], int]] = None,
          max_work: Optional[int] = None) -> Tuple[List[Request], int]:
    """The next wave: requests from the front of `pending`, in arrival order,
    while the wave holds fewer than `max_batch`, its bytes fit the budget
    beside those in flight, and (with `work`) its work -- the rows it scans --
    stays within `max_work`.  A wave's requests all complete when the wave
    does, so the work cap bounds the latency a long wave adds to its short
    requests.  A request larger than the whole budget runs alone once
    nothing else is in flight; one above the work cap runs in a wave of its
    own.  Returns (wave, its bytes)."""
    batch: List[Request] = []
    nbytes = 0
    nwork = 0
    while pending and len(batch) < max_batch:
        b = size(pending[0])
        alone = not batch and in_flight == 0
        if in_flight + nbytes + b > budget and not alone:
            break
        if work is not None and max_work is not None:
            wk = work(pending[0])
            if batch and nwork + wk > max_work:
                break
            nwork += wk
        batch.append(pending.popleft())
        nbytes += b
    return batch, nbytes


def wave_groups(batch: Sequence[Request], shared_min: int) -> Tuple[List[List[Request]], List[Request]]:
    """Splits a wave into shared passes (the count requests of one table, when
    at least `shared_min` of them are in the wave; tables in order of their
    first request, requests in arrival order) and the rest, run as one batch."""
    per_table: Dict[int, List[Request]] = {}
    for r in batch:
        if not r.proj:
            per_table.setdefault(r.table, []).append(r)
    groups = [rs for rs in per_table.values() if len(rs) >= shared_min]
    shared = {id(r) for rs in groups for r in rs}
    return groups, [r for r in batch if id(r) not in shared]


class Server:
    def __init__(self, esc, tables, mem_budget: int = 8 << 30, max_batch: int = 512, streams: int = 2,
                 device="cuda", shared_min: int = 8, compile_threads: int = 0,
                 max_wave_rows: Optional[int] = 1_200_000_000):
        self.esc = esc
        self.tables = tables
        self.budget = mem_budget
        self.max_batch = max_batch
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        # per stream: the wave's counts on the device (every library call
        # overwrites its range, so no fill is needed) and a pinned copy the
        # host reads once the wave's event has completed (no blocking read)
        self.dev_counts = [torch.empty(max_batch, dtype=torch.int64, device=self.device) for _ in range(streams)]
        self.host_counts = [torch.empty(max_batch, dtype=torch.int64, pin_memory=True) for _ in range(streams)]
        self.widths = [{n: esc.WIDTH[d] for n, d, _ in t.columns} for t in tables]
        self.in_flight_bytes = 0
        self.peak_bytes = 0
        self.waves = 0
        self.shared_min = shared_min      # count requests per table that share one pass
        self.shared_launches = 0
        self.single_launches = 0          # waves (or their remainder) of one sub-query, run as a plain call
        self.compile_threads = compile_threads
        self.max_wave_rows = max_wave_rows  # table rows a wave may scan (None: no cap)
        # per wave: launch and completion times (server clock, s), requests,
        # shared passes, table rows scanned, and how long the launch took on the host
        self.wave_log: List[dict] = []

    def _compile(self, r: Request):
        return self.esc.Predicate(self.tables[r.table], r.text, tuple(r.proj))

    def run(self, requests: Sequence[Request], clock=time.perf_counter) -> List[Request]:
        """Serves `requests` (arrival times relative to the start) and returns them completed."""
        with no_gc_pauses():
            return self._run(requests, clock)

    def _run(self, requests: Sequence[Request], clock) -> List[Request]:
        esc = self.esc
        pending: Deque[Request] = deque()
        queue = deque(sorted(requests, key=lambda r: r.arrival))
        slots: List[Optional[dict]] = [None] * len(self.streams)
        pool = _compile_pool(self.compile_threads)
        t0 = clock()
        done_n = 0
        while done_n < len(requests):
            now = clock() - t0
            while queue and queue[0].arrival <= now:
                r = queue.popleft()
                r.pred = pool.submit(self._compile, r) if pool else _Ready(self._compile(r))
                pending.append(r)
            progressed = False
            for k, st in enumerate(self.streams):
                w = slots[k]
                if w is not None and w["event"].query():
                    t_done = clock() - t0
                    w["log"]["done"] = t_done
                    counts = w["host"].tolist()
                    for r, c in zip(w["reqs"], counts):
                        r.count = int(c)
                        r.done = t_done
                    self.in_flight_bytes -= w["bytes"]
                    done_n += len(w["reqs"])
                    slots[k] = None
                    progressed = True
                if slots[k] is None and pending:
                    batch, nbytes = admit(pending, self.in_flight_bytes, self.budget, self.max_batch,
                                          lambda r: request_bytes(self.tables[r.table].nrows, r,
                                                                  self.widths[r.table]),
                                          lambda r: self.tables[r.table].nrows, self.max_wave_rows)
                    if batch:
                        t_l = clock() - t0
                        self._launch(batch, k, st, nbytes, slots)
                        slots[k]["log"].update(launch=t_l, host_s=clock() - t0 - t_l, stream=k)
                        self.wave_log.append(slots[k]["log"])
                        progressed = True
            if not progressed:
                time.sleep(0)
        if pool:
            pool.shutdown(wait=True)
        return list(requests)

    def _launch(self, batch: List[Request], k: int, st, nbytes: int, slots) -> None:
        esc = self.esc
        # shared passes first (one per table), then the rest as one batch
        groups, rest_reqs = wave_groups(batch, self.shared_min)
        batch = [r for g in groups for r in g] + rest_reqs
        nshared = len(batch) - len(rest_reqs)
        preds = []
        rows = []
        with torch.cuda.stream(st):
            # outputs are allocated on the wave's own stream, so that the
            # kernels below are ordered after their allocation
            for r in batch:
                p = r.pred.result()
                r.pred = p
                preds.append(p)
                if r.proj:
                    r.rows = p.alloc_rows(max(1, r.capacity), device=self.device)
                    rows.append(r.rows)
                else:
                    rows.append(None)
            counts = self.dev_counts[k][:len(batch)]
            i = 0
            for g in groups:
                j = i + len(g)
                esc.esc_selectivity_shared_async(self.tables[g[0].table].handle, [p.handle for p in preds[i:j]],
                                                 counts[i:j], st)
                self.shared_launches += 1
                i = j
            assert i == nshared
            if i == len(batch) - 1:
                # a lone sub-query: the plain call (less set-up than a batch of one)
                esc.esc_selectivity_async(self.tables[batch[i].table].handle, preds[i].handle, counts[i:i + 1],
                                          rows[i], st)
                self.single_launches += 1
            elif i < len(batch):
                rest = rows[i:]
                esc.esc_selectivity_batch_async([self.tables[r.table].handle for r in batch[i:]],
                                                [p.handle for p in preds[i:]], counts[i:],
                                                rest if any(x is not None for x in rest) else None, None, st)
            host = self.host_counts[k][:len(batch)]
            host.copy_(counts, non_blocking=True)   # ordered before the event on the wave's stream
            ev = torch.cuda.Event()
            ev.record(st)
        self.in_flight_bytes += nbytes
        self.peak_bytes = max(self.peak_bytes, self.in_flight_bytes)
        self.waves += 1
        log = {"requests": len(batch), "shared": len(groups),
               "rows": sum(self.tables[r.table].nrows for r in batch)}
        slots[k] = {"reqs": batch, "host": host, "event": ev, "bytes": nbytes, "preds": preds, "log": log}


@contextlib.contextmanager
def no_gc_pauses():
    """Runs a serving loop with Python's cyclic garbage collector off (one
    collection first, the previous setting restored after): a full
    collection over the loop's many small objects stops the polling thread
    for tens of milliseconds, and every request in flight waits that long.
    Memory is reclaimed by reference counting meanwhile."""
    was = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def latency_summary(reqs: Sequence[Request]) -> Dict[str, float]:
    lat = np.array([(r.done - r.arrival) * 1e3 for r in reqs])
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "throughput_per_s": len(reqs) / span}


class PlainServer:
    """One sub-query call per request, launched when it arrives (round robin
    over `streams`); the baseline that continuous batching is measured
    against.  Completion is observed by polling each request's event."""

    def __init__(self, esc, tables, streams: int = 2, device="cuda", compile_threads: int = 0):
        self.esc = esc
        self.tables = tables
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.compile_threads = compile_threads

    def run(self, requests: Sequence[Request], clock=time.perf_counter) -> List[Request]:
        with no_gc_pauses():
            return self._run(requests, clock)

    def _run(self, requests: Sequence[Request], clock) -> List[Request]:
        esc = self.esc
        queue = deque(sorted(requests, key=lambda r: r.arrival))
        pool = _compile_pool(self.compile_threads)
        inflight: Deque[tuple] = deque()
        compiling: Deque[Request] = deque()
        # count slots: each request's count on the device (the library call
        # stores it, no fill needed) and a pinned copy read once its event
        # has completed; a slot goes back to the free list then
        nslots = 1 << 15
        dev_counts = torch.empty(nslots, dtype=torch.int64, device=self.device)
        host_counts = torch.empty(nslots, dtype=torch.int64, pin_memory=True)
        host_view = host_counts.numpy()
        free = deque(range(nslots))
        t0 = clock()
        done_n, k = 0, 0
        while done_n < len(requests):
            now = clock() - t0
            progressed = False
            while queue and queue[0].arrival <= now:
                r = queue.popleft()
                if pool:
                    r.pred = pool.submit(lambda r=r: esc.Predicate(self.tables[r.table], r.text, tuple(r.proj)))
                else:
                    r.pred = _Ready(esc.Predicate(self.tables[r.table], r.text, tuple(r.proj)))
                compiling.append(r)
            while compiling and compiling[0].pred.done() and free:
                r = compiling.popleft()
                r.pred = r.pred.result()
                st = self.streams[k % len(self.streams)]
                k += 1
                s = free.popleft()
                cnt = dev_counts[s:s + 1]
                with torch.cuda.stream(st):
                    if r.proj:
                        r.rows = r.pred.alloc_rows(max(1, r.capacity), device=self.device)
                    esc.esc_selectivity_async(self.tables[r.table].handle, r.pred.handle, cnt, r.rows, st)
                    host_counts[s:s + 1].copy_(cnt, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(st)
                inflight.append((r, s, ev))
                progressed = True
            keep: Deque[tuple] = deque()
            for item in inflight:
                r, s, ev = item
                if ev.query():
                    r.count = int(host_view[s])
                    free.append(s)
                    r.done = clock() - t0
                    done_n += 1
                    progressed = True
                else:
                    keep.append(item)
            inflight = keep
            if not progressed:
                time.sleep(0)
        if pool:
            pool.shutdown(wait=True)
        return list(requests)
