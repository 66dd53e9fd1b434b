"""Autotuner for the scan's launch shape (not in the paper).

The knobs are a predicate's esc_tuning: rows staged per tile, staged bytes per
work unit and work units per SM, and the scan kernel's block shape -- its
consumer warps per CTA and the rows each lane evaluates per decoded
instruction (8 per 256-row group, one, two or four groups per pass).  Results never
depend on them; speed does, differently for small and large tables, narrow
and wide predicates, and programs with or without a udf (whose registers
limit the warps per SM).  Sub-queries are grouped into classes -- (log2 of the
table's rows, bytes per row the predicate reads, udf or not, count-only or
materialising) -- and for each class the tuner times, on a few sample
predicates (CUDA events, median of repeats), first every block shape the
class can run at the default tile and unit sizes, then every tile/unit
candidate at the fastest shape, and keeps the fastest of all.  Choices
persist in a JSON cache.

Rows per lane is 8 per group whatever the shape: lane l holds rows
64j + 2l + i of a group (j < 4, i < 2), so that each column read is one
contiguous, conflict-free run per warp for every element width.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import torch

# (max_tile_rows, max_unit_kb, units_per_sm, consumer_warps, rows_per_pass);
# block shape (0, 0) = automatic
DEFAULT = (32768, 512, 8, 0, 0)
TILE_CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (32768, 512, 8), (32768, 512, 4), (32768, 256, 16), (32768, 1024, 4),
    (8192, 512, 8), (8192, 128, 16), (4096, 256, 8), (2048, 128, 16),
)
# compiled block shapes (consumer warps, rows per lane per pass); the first
# two run programs with a udf
SHAPES_UDF: Tuple[Tuple[int, int], ...] = ((15, 16), (19, 8))
SHAPES: Tuple[Tuple[int, int], ...] = SHAPES_UDF + ((19, 16), (23, 8), (15, 32))
WIDTH = {"i32": 4, "i64": 8, "u8": 1, "u16": 2}


def read_bytes_per_row(pred) -> int:
    return sum(WIDTH[f.split()[3]] for f in pred.explain().splitlines() if f.startswith("ref "))


def has_udf(pred) -> bool:
    return any(f.split()[2] == "UDF" for f in pred.explain().splitlines() if f.startswith("instr "))


def class_key(table, pred, materialise: bool) -> str:
    u = "_u" if has_udf(pred) else ""
    return f"r{int(math.log2(max(1, table.nrows)))}_b{read_bytes_per_row(pred)}{u}_{'m' if materialise else 'c'}"


def shapes_for(key: str) -> Tuple[Tuple[int, int], ...]:
    """Block shapes a class can run: with a udf only those with the udf path."""
    return SHAPES_UDF if "_u_" in key else SHAPES


def candidates(key: str, tiles: Iterable[Tuple[int, int, int]] = TILE_CANDIDATES,
               shape: Optional[Tuple[int, int]] = None):
    """Stage 1 (shape None): every shape of the class at the default tile and
    unit sizes; stage 2: every tile/unit candidate at `shape`."""
    if shape is None:
        return [DEFAULT[:3] + sh for sh in shapes_for(key)]
    return [tuple(t) + tuple(shape) for t in tiles]


class Autotuner:
    def __init__(self, esc, cache_path: Optional[str] = None, repeats: int = 3):
        self.esc = esc
        self.cache_path = cache_path
        self.repeats = repeats
        self.cache: Dict[str, Tuple[int, ...]] = {}
        self.timings: Dict[str, Dict[str, float]] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                # entries without a block shape take the automatic one
                self.cache = {k: (tuple(v) + (0, 0))[:5] for k, v in json.load(f).items()}

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
             tiles: Iterable[Tuple[int, int, int]] = TILE_CANDIDATES) -> Dict[str, Tuple[int, ...]]:
        """Times the candidates on each class present in `preds` (all on `table`)
        that is not cached yet; returns the class -> choice map it updated."""
        tiles = tuple(tiles)
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
            times = {c: self._time(table, sample, rows, c) for c in candidates(key)}
            shape = min(times, key=times.get)[3:]
            for c in candidates(key, tiles, shape):
                if c not in times:
                    times[c] = self._time(table, sample, rows, c)
            best = min(times, key=times.get)
            self.cache[key] = best
            self.timings[key] = {str(c): t for c, t in times.items()}
            chosen[key] = best
            for p in sample:
                self.esc.esc_predicate_set_tuning(p.handle, None)
        self.save()
        return chosen

    def apply(self, table, pred, materialise: bool = False) -> Tuple[int, ...]:
        """Sets pred's launch shape to its class's choice (the default if untuned)."""
        choice = self.cache.get(class_key(table, pred, materialise), DEFAULT)
        self.esc.esc_predicate_set_tuning(pred.handle, choice)
        return choice
