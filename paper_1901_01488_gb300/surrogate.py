"""Learned selectivity surrogate, trained on and evaluated against exact ESC.

Not in the paper: the paper computes every selectivity exactly (Sec. 2).
This module adds a small network that *estimates* log10 selectivity from
the compiled predicate, trained on (predicate, exact count) pairs that ESC
itself produces; exact ESC stays the reference (q-error) and the fallback,
and is the only source of counts a planner may treat as exact.

* Synopsis: per-column statistics of a table sample (sorted values), the
  estimator ESC replaces.  `Synopsis.independence(listing)` evaluates a
  compiled program (its listing from esc_predicate_explain: the merged,
  domain-clamped tests the kernel runs) with each test's sample selectivity,
  AND as a product, OR as a + b - ab, NOT as 1 - a.
* `Synopsis.features(listing)`: 64 features from the same listing -- for
  each of 8 column slots [tested, log10 of its tests' sample selectivity,
  lo, hi (normalised to the column's sample range), set size / 16, under an
  OR, udf operand] (7 per slot), and 8 global ones (log10 of the
  independence estimate, tests, ORs, NOTs, udf, set tests).  The network learns the
  correction independence misses (correlated columns, udf terms).
* Surrogate: the MLP 64 -> 128 -> 128 -> 1 of libesc (esc_mlp_forward,
  esc_mlp_grad, esc_mlp_adam); float32 master weights, bfloat16 copies.
* `Fallback`: the surrogate where its held-out error is small (calibrated
  per predicted-selectivity bucket), exact ESC otherwise.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

NFEAT = 64
NSLOT = 8
PER_SLOT = 7
LOG_FLOOR = -8.0          # log10 selectivity floor of the features (an empty test)


def _parse(listing: str):
    """(ref slot -> column name, instructions as token lists) of a program listing."""
    refs, code = {}, []
    for line in listing.splitlines():
        f = line.split()
        if not f:
            continue
        if f[0] == "ref":
            refs[int(f[1])] = f[2]
        elif f[0] == "instr":
            code.append(f[2:])
    return refs, code


class Synopsis:
    """Per-column statistics of a table sample (every value kept, sorted):
    the selectivity of a range, an equality or a set on one column, exact on
    the sample."""

    def __init__(self, host_cols: Dict[str, np.ndarray], slots: Sequence[str]):
        self.slots = list(slots)[:NSLOT]
        self.sorted = {c: np.sort(np.asarray(a).astype(np.int64)) for c, a in host_cols.items()}
        self.n = len(next(iter(self.sorted.values())))
        self.lo = {c: int(v[0]) if len(v) else 0 for c, v in self.sorted.items()}
        self.hi = {c: int(v[-1]) if len(v) else 0 for c, v in self.sorted.items()}

    def range_sel(self, c: str, a: int, b: int) -> float:
        if a > b or self.n == 0:
            return 0.0
        v = self.sorted[c]
        return float(np.searchsorted(v, b, "right") - np.searchsorted(v, a, "left")) / self.n

    def set_sel(self, c: str, vals: Sequence[int]) -> float:
        return min(1.0, sum(self.range_sel(c, v, v) for v in set(vals)))

    @staticmethod
    def udf_sel(m: int, a: int, b: int) -> float:
        """Remainders of non-negative products taken as uniform on 0..m-1."""
        lo, hi = max(a, 0), min(b, m - 1)
        return max(0, hi - lo + 1) / m

    def _test(self, refs, ins) -> Tuple[float, Optional[str], dict]:
        op = ins[0]
        if op == "RANGE":
            c = refs[int(ins[1])]
            return self.range_sel(c, int(ins[3]), int(ins[4])), c, {"lo": int(ins[3]), "hi": int(ins[4])}
        if op == "IN":
            c = refs[int(ins[1])]
            vals = [int(v) for v in ins[3].split(",")] if len(ins) > 3 else []
            return self.set_sel(c, vals), c, {"lo": min(vals, default=0), "hi": max(vals, default=0),
                                              "set": len(vals)}
        if op == "UDF":
            c, c2 = refs[int(ins[1])], refs[int(ins[3])]
            return self.udf_sel(int(ins[5]), int(ins[6]), int(ins[7])), c, {"udf": c2}
        return 0.0, None, {}

    def _walk(self, listing: str):
        """Evaluates the program on selectivities; also collects, per column,
        the tests it makes (with whether they sit under an OR)."""
        refs, code = _parse(listing)
        stack: List[Tuple[float, List[int]]] = []   # (selectivity, indices of the tests below)
        tests = []                                   # (column, selectivity, info, under_or)
        nor = nnot = 0
        for ins in code:
            op = ins[0]
            if op in ("RANGE", "IN", "UDF"):
                sel, c, info = self._test(refs, ins)
                tests.append([c, sel, info, False])
                stack.append((sel, [len(tests) - 1]))
            elif op == "TRUE":
                stack.append((1.0, []))
            elif op == "FALSE":
                stack.append((0.0, []))
            elif op == "NOT":
                a, ta = stack.pop()
                stack.append((1.0 - a, ta))
                nnot += 1
            elif op in ("AND", "OR"):
                b, tb = stack.pop()
                a, ta = stack.pop()
                if op == "AND":
                    stack.append((a * b, ta + tb))
                else:
                    for t in ta + tb:
                        tests[t][3] = True
                    stack.append((a + b - a * b, ta + tb))
                    nor += 1
            # JZ / JNZ only skip work whose result is decided: no effect on the value
        sel = stack[-1][0] if stack else 1.0
        return min(1.0, max(0.0, sel)), tests, nor, nnot

    def independence(self, listing: str) -> float:
        return self._walk(listing)[0]

    def features(self, listing: str) -> np.ndarray:
        """Per slot: [tested, log10 of its tests' selectivity (sample, as if
        independent), lo, hi (of its range / set tests, normalised to the
        column's sample range), set size / 16, under an OR, udf operand];
        then [log10 of the independence estimate, tests / 8, ORs / 4,
        NOTs / 4, has a udf, set tests / 4, 0, 0].  Logs are scaled by 1/8."""
        sel, tests, nor, nnot = self._walk(listing)
        f = np.zeros(NFEAT, dtype=np.float32)

        def lg(x):
            return max(LOG_FLOOR, math.log10(max(x, 1e-300))) / -LOG_FLOOR

        per: Dict[str, List] = {}
        for c, s_, info, under_or in tests:
            per.setdefault(c, []).append((s_, info, under_or))
            if "udf" in info and info["udf"] in self.slots:
                f[PER_SLOT * self.slots.index(info["udf"]) + 6] = 1.0
        for c, lst in per.items():
            if c not in self.slots:
                continue
            b = PER_SLOT * self.slots.index(c)
            span = max(1, self.hi[c] - self.lo[c])
            prod, lo, hi = 1.0, 1.0, 0.0
            for s_, info, under_or in lst:
                prod *= s_
                if "lo" in info:
                    lo = min(lo, (info["lo"] - self.lo[c]) / span)
                    hi = max(hi, (info["hi"] - self.lo[c]) / span)
                if "set" in info:
                    f[b + 4] = max(f[b + 4], info["set"] / 16.0)
                if "udf" in info:
                    f[b + 6] = 1.0
                if under_or:
                    f[b + 5] = 1.0
            f[b + 0] = 1.0
            f[b + 1] = lg(prod)
            if hi >= lo:
                f[b + 2] = min(1.0, max(0.0, lo))
                f[b + 3] = min(1.0, max(0.0, hi))
        g = PER_SLOT * NSLOT
        f[g + 0] = lg(sel)
        f[g + 1] = len(tests) / 8.0
        f[g + 2] = nor / 4.0
        f[g + 3] = nnot / 4.0
        f[g + 4] = float(any("udf" in t[2] for t in tests))
        f[g + 5] = float(sum(1 for t in tests if "set" in t[2])) / 4.0
        return f

    def features_batch(self, listings: Sequence[str]) -> np.ndarray:
        if not listings:
            return np.zeros((0, NFEAT), np.float32)
        return np.stack([self.features(l) for l in listings])

    def base_log(self, listings: Sequence[str], nrows: int) -> np.ndarray:
        """log10 selectivity of the independence estimate, clamped like a
        label (at least one row): the network learns the correction to it."""
        est = np.array([self.independence(l) for l in listings], dtype=np.float64) * nrows
        return log_selectivity(est, nrows)


def to_bf16(x: np.ndarray, device) -> torch.Tensor:
    """float32 array -> bfloat16 bit patterns (int16 tensor) on `device`."""
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(device).to(torch.bfloat16).view(torch.int16)


def log_selectivity(counts: np.ndarray, nrows: int) -> np.ndarray:
    """log10 of the selectivity, counts clamped to at least one row."""
    return np.log10(np.maximum(np.asarray(counts, dtype=np.float64), 1.0) / float(nrows)).astype(np.float32)


def qerror(est: np.ndarray, true: np.ndarray) -> np.ndarray:
    """max(est/true, true/est), both counts clamped to at least one row."""
    e = np.maximum(np.asarray(est, dtype=np.float64), 1.0)
    t = np.maximum(np.asarray(true, dtype=np.float64), 1.0)
    return np.maximum(e / t, t / e)


def exact_counts(esc, table, texts: Sequence[str], chunk: int = 2048, stream=None) -> np.ndarray:
    """Exact ESC counts of many predicates on one table: each chunk compiled
    in one call (host threads), one shared pass per chunk
    (esc_selectivity_shared_async), counts read back once at the end."""
    n = len(texts)
    dev = torch.zeros(max(1, n), dtype=torch.int64, device="cuda")
    keep = []
    for s in range(0, n, chunk):
        ps = esc.PredicateSet(table, list(texts[s:s + chunk]))
        esc.esc_selectivity_shared_async(table.handle, ps.handles, dev[s:s + len(ps)], stream=stream)
        keep.append(ps)  # predicates stay alive until their pass has run
    return dev[:n].cpu().numpy().astype(np.int64)


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
            lr: float = 2e-3, seed: int = 1, lr_end: Optional[float] = None) -> List[float]:
        """Minibatch Adam on mean squared error; returns the mean loss per epoch.
        With `lr_end` the step size falls from `lr` to `lr_end` along a half
        cosine over the steps of the run (less noise in the final weights)."""
        n = x_bf16.shape[0]
        grad = torch.zeros_like(self.params)
        lsum = torch.zeros(1, dtype=torch.float32, device=self.device)
        gen = torch.Generator(device=self.device).manual_seed(seed)
        curve = []
        steps = epochs * ((n + batch - 1) // batch)
        k = 0
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
                rate = lr
                if lr_end is not None:
                    rate = lr_end + (lr - lr_end) * 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps - 1)))
                k += 1
                self.esc.esc_mlp_adam(self.params, self.wbf, grad, self.m, self.v, rate, self.step)
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


def listings(esc, table, texts: Sequence[str], chunk: int = 4096) -> List[str]:
    """Program listings of many predicates (compiled in one call per chunk)."""
    out: List[str] = []
    for s in range(0, len(texts), chunk):
        ps = esc.PredicateSet(table, list(texts[s:s + chunk]))
        out.extend(esc.esc_predicate_explain(h) for h in ps.handles)
        ps.close()
    return out


class Fallback:
    """Estimates with exact ESC as the fallback: the surrogate's estimate
    (base + the network's correction, in log10 selectivity) is used where the
    calibration set says its q-error stays within `tol` for `coverage` of the
    predicates of that predicted-selectivity decade; elsewhere the count comes
    from exact ESC."""

    def __init__(self, model: "Surrogate", tol: float = 2.0, coverage: float = 0.95):
        self.model = model
        self.tol = tol
        self.coverage = coverage
        self.trusted: Dict[int, bool] = {}

    @staticmethod
    def bucket(log_sel: float) -> int:
        return int(math.floor(max(LOG_FLOOR, min(0.0, log_sel))))

    def predict_log(self, x_bf16: torch.Tensor, base: np.ndarray) -> np.ndarray:
        return base + self.model.predict(x_bf16).cpu().numpy().astype(np.float64)

    def calibrate(self, x_bf16: torch.Tensor, base: np.ndarray, counts: np.ndarray, nrows: int) -> Dict[int, bool]:
        pred = self.predict_log(x_bf16, base)
        q = qerror(10.0 ** pred * nrows, counts)
        for b in set(self.bucket(v) for v in pred):
            sel = np.array([self.bucket(v) == b for v in pred])
            self.trusted[b] = bool(sel.sum() >= 20 and np.mean(q[sel] <= self.tol) >= self.coverage)
        return self.trusted

    def estimate(self, x_bf16: torch.Tensor, base: np.ndarray, exact_fn, nrows: int) -> Tuple[np.ndarray, np.ndarray]:
        """(row estimates, used_exact mask): exact_fn(indices) -> exact counts."""
        pred = self.predict_log(x_bf16, base)
        use_exact = np.array([not self.trusted.get(self.bucket(v), False) for v in pred])
        est = 10.0 ** pred * nrows
        idx = np.flatnonzero(use_exact)
        if len(idx):
            est[idx] = np.asarray(exact_fn(idx), dtype=np.float64)
        return est, use_exact
