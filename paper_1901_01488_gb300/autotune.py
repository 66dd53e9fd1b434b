"""Autotuner for the scan's launch shape (not in the paper).

The knobs are a predicate's esc_tuning: rows staged per tile, staged bytes per
work unit, and work units per SM.  Results never depend on them; speed does,
differently for small and large tables and for narrow and wide predicates.
Sub-queries are grouped into classes -- (log2 of the table's rows, bytes per
row the predicate reads, count-only or materialising) -- and for each class
the tuner times every candidate on a few sample predicates (CUDA events,
median of repeats) and keeps the fastest.  Choices persist in a JSON cache.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import torch

DEFAULT = (32768, 512, 8)
CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (32768, 512, 8), (32768, 512, 4), (32768, 256, 16), (32768, 1024, 4),
    (8192, 512, 8), (8192, 128, 16), (4096, 256, 8), (2048, 128, 16),
)
WIDTH = {"i32": 4, "i64": 8, "u8": 1, "u16": 2}


def read_bytes_per_row(pred) -> int:
    return sum(WIDTH[f.split()[3]] for f in pred.explain().splitlines() if f.startswith("ref "))


def class_key(table, pred, materialise: bool) -> str:
    return f"r{int(math.log2(max(1, table.nrows)))}_b{read_bytes_per_row(pred)}_{'m' if materialise else 'c'}"


class Autotuner:
    def __init__(self, esc, cache_path: Optional[str] = None, repeats: int = 3):
        self.esc = esc
        self.cache_path = cache_path
        self.repeats = repeats
        self.cache: Dict[str, Tuple[int, int, int]] = {}
        self.timings: Dict[str, Dict[str, float]] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = {k: tuple(v) for k, v in json.load(f).items()}

    def save(self) -> None:
        if self.cache_path:
            with open(self.cache_path, "w") as f:
                json.dump({k: list(v) for k, v in self.cache.items()}, f, indent=1, sort_keys=True)

    def _time(self, table, preds, rows, cand) -> float:
        esc = self.esc
        for p in preds:
            esc.esc_predicate_set_tuning(p.handle, cand)
        dc = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.cuda.current_stream()

        def run():
            for p, r in zip(preds, rows):
                esc.esc_selectivity_async(table.handle, p.handle, dc, r, st)

        run()
        torch.cuda.synchronize()
        samples = []
        for _ in range(self.repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            run()
            b.record(st)
            torch.cuda.synchronize()
            samples.append(a.elapsed_time(b))
        return statistics.median(samples)

    def tune(self, table, preds: Sequence, materialise: bool = False,
             candidates: Iterable[Tuple[int, int, int]] = CANDIDATES) -> Dict[str, Tuple[int, int, int]]:
        """Times the candidates on each class present in `preds` (all on `table`)
        that is not cached yet; returns the class -> choice map it updated."""
        by_class: Dict[str, List] = {}
        for p in preds:
            by_class.setdefault(class_key(table, p, materialise), []).append(p)
        chosen = {}
        for key, ps in by_class.items():
            if key in self.cache:
                continue
            sample = ps[:4]
            rows = []
            for p in sample:
                if materialise:
                    n = self.esc.count(table, p)
                    rows.append(p.alloc_rows(max(1, n)))
                else:
                    rows.append(None)
            times = {c: self._time(table, sample, rows, c) for c in candidates}
            best = min(times, key=times.get)
            self.cache[key] = best
            self.timings[key] = {str(c): t for c, t in times.items()}
            chosen[key] = best
            for p in sample:
                self.esc.esc_predicate_set_tuning(p.handle, None)
        self.save()
        return chosen

    def apply(self, table, pred, materialise: bool = False) -> Tuple[int, int, int]:
        """Sets pred's launch shape to its class's choice (the default if untuned)."""
        choice = self.cache.get(class_key(table, pred, materialise), DEFAULT)
        self.esc.esc_predicate_set_tuning(pred.handle, choice)
        return choice
