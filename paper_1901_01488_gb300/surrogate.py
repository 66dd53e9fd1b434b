"""Learned selectivity surrogate, trained on and evaluated against exact ESC.

Not in the paper: the paper computes every selectivity exactly (Sec. 2).
This module adds a small network that *estimates* log10 selectivity from
the predicate alone, trained on (predicate, exact count) pairs that ESC
itself produces; exact ESC stays the reference (q-error) and the fallback, and
is the only source of counts a planner may treat as exact.

* encode(): 64 features = 8 column slots x [present, lo, hi, is_eq, is_in,
  in_size / 16, in_or_pair, is_udf], bounds normalised to the column domain.
* Surrogate: the MLP 64 -> 128 -> 128 -> 1 of libesc (esc_mlp_forward,
  esc_mlp_grad, esc_mlp_adam); float32 master weights, bfloat16 copies.
* independence_estimate(): the synopsis approach ESC replaces (per-column
  histograms combined under independence), as the comparison point.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np
import torch

from . import datagen

NFEAT = 64
SLOTS = datagen.SKEWED_COLUMNS          # key, code150, code25, code7, day, price, qty, key2


def _norm(col: str, v: float) -> float:
    _, lo, hi = datagen.SKEWED_SCHEMA[col]
    return min(1.0, max(0.0, (v - lo) / max(1, hi - lo)))


def encode(pred: datagen.Predicate) -> np.ndarray:
    f = np.zeros(NFEAT, dtype=np.float32)
    have = np.zeros(len(SLOTS), dtype=bool)

    def put(t: datagen.Term, in_or: bool):
        if t.kind == "udf":
            s = SLOTS.index("price")
            lo, hi = (t.lo + 1) / datagen.UDF_MODULUS, 1.0
        elif t.kind == "in":
            s = SLOTS.index(t.col)
            lo, hi = _norm(t.col, min(t.values)), _norm(t.col, max(t.values))
        else:
            s = SLOTS.index(t.col)
            lo, hi = _norm(t.col, t.lo), _norm(t.col, t.hi if t.kind == "range" else t.lo)
        b = 8 * s
        if have[s]:                       # several terms on one column: intersect
            lo, hi = max(lo, f[b + 1]), min(hi, f[b + 2])
        have[s] = True
        f[b + 0] = 1.0
        f[b + 1], f[b + 2] = lo, hi
        f[b + 3] = max(f[b + 3], float(t.kind == "eq"))
        f[b + 4] = max(f[b + 4], float(t.kind == "in"))
        f[b + 5] = max(f[b + 5], len(t.values) / 16.0)
        f[b + 6] = max(f[b + 6], float(in_or))
        f[b + 7] = max(f[b + 7], float(t.kind == "udf"))

    for t in pred.terms:
        if t.kind == "or":
            for part in t.parts:
                put(part, True)
        else:
            put(t, False)
    return f


def encode_batch(preds: Sequence[datagen.Predicate]) -> np.ndarray:
    return np.stack([encode(p) for p in preds]) if preds else np.zeros((0, NFEAT), np.float32)


def to_bf16(x: np.ndarray, device) -> torch.Tensor:
    """float32 array -> bfloat16 bit patterns (int16 tensor) on `device`."""
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(device).to(torch.bfloat16).view(torch.int16)


def log_selectivity(counts: np.ndarray, nrows: int) -> np.ndarray:
    return np.log10(np.maximum(counts, 1) / float(nrows)).astype(np.float32)


def qerror(est: np.ndarray, true: np.ndarray) -> np.ndarray:
    """max(est/true, true/est), both counts clamped to at least one row."""
    e = np.maximum(np.asarray(est, dtype=np.float64), 1.0)
    t = np.maximum(np.asarray(true, dtype=np.float64), 1.0)
    return np.maximum(e / t, t / e)


def exact_counts(esc, table, preds: Sequence[datagen.Predicate], chunk: int = 2048, stream=None) -> np.ndarray:
    """Exact ESC counts of many predicates on one table: each chunk compiled
    in one call (host threads), one shared pass per chunk
    (esc_selectivity_shared_async), counts read back once at the end."""
    n = len(preds)
    dev = torch.zeros(max(1, n), dtype=torch.int64, device="cuda")
    keep = []
    for s in range(0, n, chunk):
        ps = esc.PredicateSet(table, [p.text for p in preds[s:s + chunk]])
        esc.esc_selectivity_shared_async(table.handle, ps.handles, dev[s:s + len(ps)], stream=stream)
        keep.append(ps)  # predicates stay alive until their pass has run
    out = dev[:n].cpu().numpy().astype(np.int64)
    return out


class Surrogate:
    """The MLP with Adam state, all on one CUDA device, trained by libesc kernels."""

    def __init__(self, esc, device="cuda", seed: int = 0):
        self.esc = esc
        self.device = torch.device(device)
        g = torch.Generator().manual_seed(seed)
        p = torch.zeros(esc.MLP_PARAMS, dtype=torch.float32)
        o = 0
        for rows, cols in ((128, 64), (128, 1), (128, 128), (128, 1), (128, 1), (1, 1)):
            n = rows * cols
            if cols > 1:                                     # He initialisation
                p[o:o + n] = torch.randn(n, generator=g) * math.sqrt(2.0 / cols)
            o += n
        p[24832:24960] = torch.randn(128, generator=g) * math.sqrt(1.0 / 128)   # w3
        self.params = p.to(self.device)
        self.wbf = self.params.to(torch.bfloat16).view(torch.int16).contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0

    def predict(self, x_bf16: torch.Tensor) -> torch.Tensor:
        y = torch.empty(x_bf16.shape[0], dtype=torch.float32, device=self.device)
        self.esc.esc_mlp_forward(x_bf16, self.wbf, self.params, y)
        return y

    def fit(self, x_bf16: torch.Tensor, y: torch.Tensor, epochs: int = 20, batch: int = 4096,
            lr: float = 2e-3, seed: int = 1) -> List[float]:
        """Minibatch Adam on mean squared error; returns the mean loss per epoch."""
        n = x_bf16.shape[0]
        grad = torch.zeros_like(self.params)
        lsum = torch.zeros(1, dtype=torch.float32, device=self.device)
        gen = torch.Generator(device=self.device).manual_seed(seed)
        curve = []
        for _ in range(epochs):
            perm = torch.randperm(n, device=self.device, generator=gen)
            lsum.zero_()
            for s in range(0, n, batch):
                idx = perm[s:s + batch]
                xb = x_bf16[idx].contiguous()
                yb = y[idx].contiguous()
                grad.zero_()
                self.esc.esc_mlp_grad(xb, yb, self.wbf, self.params, grad, lsum)
                self.step += 1
                self.esc.esc_mlp_adam(self.params, self.wbf, grad, self.m, self.v, lr, self.step)
            curve.append(float(lsum.item()) / n)
        return curve

    def state_dict(self) -> Dict[str, torch.Tensor]:
        return {"params": self.params.cpu(), "m": self.m.cpu(), "v": self.v.cpu(),
                "step": torch.tensor(self.step)}

    def load_state_dict(self, st: Dict[str, torch.Tensor]) -> None:
        self.params = st["params"].to(self.device).contiguous()
        self.wbf = self.params.to(torch.bfloat16).view(torch.int16).contiguous()
        self.m = st["m"].to(self.device).contiguous()
        self.v = st["v"].to(self.device).contiguous()
        self.step = int(st["step"])


# ---------------------------------------------------------------- synopsis baseline
class Histograms:
    """Per-column statistics of a table sample: exact frequencies for columns
    with at most 2^24 values, used under the independence assumption."""

    def __init__(self, host_cols: Dict[str, np.ndarray]):
        self.n = len(next(iter(host_cols.values())))
        self.freq = {}
        for c, a in host_cols.items():
            kind, lo, hi = datagen.SKEWED_SCHEMA[c]
            if hi - lo < (1 << 24) + 1:
                self.freq[c] = np.cumsum(np.bincount(a.astype(np.int64) - lo, minlength=hi - lo + 1)) / self.n
            else:                                            # wide: 4096 equal-width buckets
                edges = np.linspace(lo, hi + 1, 4097)
                h, _ = np.histogram(a, bins=edges)
                self.freq[c] = (edges, np.cumsum(h) / self.n)

    def range_sel(self, c: str, a: int, b: int) -> float:
        _, lo, hi = datagen.SKEWED_SCHEMA[c]
        a, b = max(a, lo), min(b, hi)
        if a > b:
            return 0.0
        f = self.freq[c]
        if isinstance(f, tuple):
            edges, cum = f
            def at(x):   # fraction of rows <= x, linear inside a bucket
                i = int(np.searchsorted(edges, x, side="right")) - 1
                i = min(max(i, 0), len(cum) - 1)
                prev = cum[i - 1] if i > 0 else 0.0
                return prev + (cum[i] - prev) * (x + 1 - edges[i]) / (edges[i + 1] - edges[i])
            return max(0.0, at(b) - at(a - 1))
        return float(f[b - lo] - (f[a - lo - 1] if a > lo else 0.0))

    def term_sel(self, t: datagen.Term) -> float:
        if t.kind == "eq":
            return self.range_sel(t.col, t.lo, t.lo)
        if t.kind == "range":
            return self.range_sel(t.col, t.lo, t.hi)
        if t.kind == "in":
            return min(1.0, sum(self.range_sel(t.col, v, v) for v in set(t.values)))
        if t.kind == "udf":
            m = datagen.UDF_MODULUS
            return (m - 1 - t.lo) / m
        a, b = self.term_sel(t.parts[0]), self.term_sel(t.parts[1])
        return a + b - a * b


def independence_estimate(h: Histograms, pred: datagen.Predicate) -> float:
    s = 1.0
    for t in pred.terms:
        s *= h.term_sel(t)
    return s
