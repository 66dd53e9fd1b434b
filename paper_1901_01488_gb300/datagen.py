"""Seeded synthetic inputs: tables and predicates.

This module only draws random numbers and lays them out as columns and as
predicate texts.  It evaluates no predicate and counts nothing: the method's
arithmetic lives in the CUDA library (the product) and in ``oracle/`` (the
checker), and both are fed the exact same bytes produced here.

Random numbers come from a counter-based generator: the SplitMix64 finalizer
of Steele, Lea and Flood ("Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to ``key(seed, stream) + (i + 1) * gamma``.  Every element
``i`` of every column is therefore a pure function of (seed, stream, i), so a
table is identical whether it is generated on the CPU or on a GPU, and in any
chunking.  All arithmetic below is int64 with two's-complement wrap-around and
masked (logical) right shifts, which torch implements identically on both
devices; the uint64 cross-check lives in the tests.

Workload shapes (stand-ins for the paper's TPC-H / SSB workloads of Sec. 3,
which are not reproduced):

* ``single_table`` -- 1,000,000 rows: key i32 U[0, 2^20), day i32 U[0, 2556],
  price i64 U[100, 10^7], category u8 U{0..24}.
* ``skewed_table`` -- 60,000,000 rows x 8 columns, 32 B/row: Zipf(1.1) keys
  over 2^24, dictionary codes of 150 / 25 / 7 values with
  code25 = code150 mod 25 on 70 % of rows, day, price, qty, a second key.
* ``star_schema`` -- a 600,000,000-row fact table of 4 Zipf(0.8) foreign keys
  into dense-key dimensions of 2,000,000 / 200,000 / 30,000 / 2,556 rows plus
  2 measures, and the dimension tables (3 attributes each).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(u: int) -> int:
    """Python int in [0, 2^64) -> the int64 with the same bit pattern."""
    u &= MASK64
    return u - (1 << 64) if u >= (1 << 63) else u


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor by k (1 <= k <= 63)."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _mix_py(z: int) -> int:
    """SplitMix64 finalizer on a Python int (used only to derive stream keys)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return _mix_py(_mix_py(seed * GAMMA + 0x5851F42D4C957F2D) + stream * 0xD1B54A32D192ED03)


def raw_u64(seed: int, stream: int, start: int, count: int, device) -> torch.Tensor:
    """Elements start..start+count-1 of stream (seed, stream), as int64 bit patterns."""
    key = _s64(stream_key(seed, stream))
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = i * _s64(GAMMA) + key
    z = (z ^ _srl(z, 30)) * _s64(_M1)
    z = (z ^ _srl(z, 27)) * _s64(_M2)
    return z ^ _srl(z, 31)


def uniform_int(raw: torch.Tensor, lo: int, hi: int) -> torch.Tensor:
    """Map raw 64-bit draws to integers in [lo, hi] (hi - lo < 2^32) by the high 32 bits."""
    span = hi - lo + 1
    assert 1 <= span <= (1 << 32)
    return lo + _srl(_srl(raw, 32) * span, 32)


def uniform_01(raw: torch.Tensor) -> torch.Tensor:
    """Map raw draws to float64 in [0, 1) using the top 53 bits."""
    return _srl(raw, 11).to(torch.float64) * (2.0 ** -53)


# ---------------------------------------------------------------- Zipf ranks
_ZIPF_CACHE: Dict[Tuple[float, int, str], torch.Tensor] = {}


def zipf_cdf(s: float, n: int, device) -> torch.Tensor:
    """Normalised cumulative weights of P(rank r) ~ r^-s, r = 1..n (float64)."""
    k = (float(s), int(n), str(device))
    if k not in _ZIPF_CACHE:
        r = np.arange(1, n + 1, dtype=np.float64)
        c = np.cumsum(r ** (-float(s)))
        c /= c[-1]
        _ZIPF_CACHE[k] = torch.from_numpy(c).to(device)
    return _ZIPF_CACHE[k]


def zipf_probabilities(s: float, n: int) -> np.ndarray:
    r = np.arange(1, n + 1, dtype=np.float64)
    w = r ** (-float(s))
    return w / w.sum()


ZIPF_MULT = 1_000_003  # prime: (a*r + b) mod n is a bijection for every n it does not divide


def zipf_key_of_rank(rank0: torch.Tensor, n: int, salt: int) -> torch.Tensor:
    """Seeded bijection of 0-based ranks onto [0, n): popular keys are scattered."""
    assert math.gcd(ZIPF_MULT, n) == 1
    return (rank0 * ZIPF_MULT + (salt % n)) % n


def zipf_keys(seed: int, stream: int, start: int, count: int, s: float, n: int,
              device, salt: int = 12345) -> torch.Tensor:
    cdf = zipf_cdf(s, n, device)
    u = uniform_01(raw_u64(seed, stream, start, count, device))
    rank0 = torch.searchsorted(cdf, u, right=True).clamp_(max=n - 1)
    return zipf_key_of_rank(rank0, n, salt)


# ---------------------------------------------------------------- tables
DTYPES = ("i32", "i64", "u8", "u16")
WIDTH = {"i32": 4, "i64": 8, "u8": 1, "u16": 2}
_TORCH = {"i32": torch.int32, "i64": torch.int64, "u8": torch.uint8, "u16": torch.int16}
_NUMPY = {"i32": np.int32, "i64": np.int64, "u8": np.uint8, "u16": np.uint16}
DOMAIN = {"i32": (-(1 << 31), (1 << 31) - 1), "i64": (-(1 << 63), (1 << 63) - 1),
          "u8": (0, 255), "u16": (0, 65535)}


def to_storage(v: torch.Tensor, dtype: str) -> torch.Tensor:
    """int64 values -> the column's storage tensor (u16 kept as int16 bit patterns)."""
    if dtype == "u16":
        v = torch.where(v >= 32768, v - 65536, v)
    return v.to(_TORCH[dtype])


@dataclasses.dataclass
class Column:
    name: str
    dtype: str           # one of DTYPES
    data: torch.Tensor   # storage tensor, one element per row

    def numpy(self) -> np.ndarray:
        a = self.data.detach().cpu().numpy()
        return a.view(_NUMPY[self.dtype])


@dataclasses.dataclass
class Table:
    nrows: int
    columns: List[Column]

    def col(self, name: str) -> Column:
        for c in self.columns:
            if c.name == name:
                return c
        raise KeyError(name)

    def host(self) -> Dict[str, np.ndarray]:
        return {c.name: c.numpy() for c in self.columns}

    def to(self, device) -> "Table":
        return Table(self.nrows, [Column(c.name, c.dtype, c.data.to(device)) for c in self.columns])

    @property
    def row_bytes(self) -> int:
        return sum(WIDTH[c.dtype] for c in self.columns)


def _chunks(n: int, chunk: int):
    s = 0
    while s < n:
        yield s, min(chunk, n - s)
        s += chunk


def _fill(nrows: int, dtype: str, device, fn, chunk: int = 1 << 25) -> torch.Tensor:
    out = torch.empty(nrows, dtype=_TORCH[dtype], device=device)
    for s, c in _chunks(nrows, chunk):
        out[s:s + c] = to_storage(fn(s, c), dtype)
    return out


SINGLE_TABLE_PREDICATE = ("category = 7 AND day BETWEEN 400 AND 765 AND "
                          "(price = 50000 OR price > 9000000)")
SINGLE_TABLE_PROJECTION = ("key", "day", "price")


def single_table(nrows: int = 1_000_000, seed: int = 1, device="cpu") -> Table:
    """Plain one-table workload: key, day, price, category (uniform)."""
    cols = [
        Column("key", "i32", _fill(nrows, "i32", device,
               lambda s, c: uniform_int(raw_u64(seed, 0, s, c, device), 0, (1 << 20) - 1))),
        Column("day", "i32", _fill(nrows, "i32", device,
               lambda s, c: uniform_int(raw_u64(seed, 1, s, c, device), 0, 2556))),
        Column("price", "i64", _fill(nrows, "i64", device,
               lambda s, c: uniform_int(raw_u64(seed, 2, s, c, device), 100, 10_000_000))),
        Column("category", "u8", _fill(nrows, "u8", device,
               lambda s, c: uniform_int(raw_u64(seed, 3, s, c, device), 0, 24))),
    ]
    return Table(nrows, cols)


SKEWED_KEY_SPACE = 1 << 24
SKEWED_ZIPF_S = 1.1


def skewed_table(nrows: int = 60_000_000, seed: int = 2, device="cpu") -> Table:
    """Skewed / correlated fact table, 32 bytes per row."""
    n = SKEWED_KEY_SPACE

    def code25(s, c):
        c150 = uniform_int(raw_u64(seed, 1, s, c, device), 0, 149)
        corr = uniform_01(raw_u64(seed, 2, s, c, device)) < 0.7
        indep = uniform_int(raw_u64(seed, 3, s, c, device), 0, 24)
        return torch.where(corr, c150 % 25, indep)

    cols = [
        Column("key", "i32", _fill(nrows, "i32", device,
               lambda s, c: zipf_keys(seed, 0, s, c, SKEWED_ZIPF_S, n, device, salt=777))),
        Column("code150", "u16", _fill(nrows, "u16", device,
               lambda s, c: uniform_int(raw_u64(seed, 1, s, c, device), 0, 149))),
        Column("code25", "u8", _fill(nrows, "u8", device, code25)),
        Column("code7", "u8", _fill(nrows, "u8", device,
               lambda s, c: uniform_int(raw_u64(seed, 4, s, c, device), 0, 6))),
        Column("day", "i32", _fill(nrows, "i32", device,
               lambda s, c: uniform_int(raw_u64(seed, 5, s, c, device), 0, 2556))),
        Column("price", "i64", _fill(nrows, "i64", device,
               lambda s, c: uniform_int(raw_u64(seed, 6, s, c, device), 100, 10_000_000))),
        Column("qty", "i64", _fill(nrows, "i64", device,
               lambda s, c: uniform_int(raw_u64(seed, 7, s, c, device), 1, 50))),
        Column("key2", "i32", _fill(nrows, "i32", device,
               lambda s, c: zipf_keys(seed, 8, s, c, SKEWED_ZIPF_S, n, device, salt=4242))),
    ]
    return Table(nrows, cols)


# Column domains of the skewed table, as the predicate generator sees them.
# kind: 'uniform' (integers lo..hi equally likely), 'code' (K codes 0..K-1),
# 'zipf' (Zipf keys over [0, n)).
SKEWED_SCHEMA = {
    "key": ("zipf", 0, SKEWED_KEY_SPACE - 1),
    "code150": ("code", 0, 149),
    "code25": ("code", 0, 24),
    "code7": ("code", 0, 6),
    "day": ("uniform", 0, 2556),
    "price": ("uniform", 100, 10_000_000),
    "qty": ("uniform", 1, 50),
    "key2": ("zipf", 0, SKEWED_KEY_SPACE - 1),
}
SKEWED_COLUMNS = tuple(SKEWED_SCHEMA)
SKEWED_PROJECTION = ("key", "day", "price")
UDF_MODULUS = 97


# ---------------------------------------------------------------- predicates
@dataclasses.dataclass
class Term:
    kind: str                 # 'eq' | 'range' | 'in' | 'or' | 'udf'
    col: str = ""
    lo: int = 0
    hi: int = 0
    values: Tuple[int, ...] = ()
    parts: Tuple["Term", ...] = ()   # for 'or'
    est: float = 1.0          # selectivity the generator aimed at (not a count)

    def text(self) -> str:
        if self.kind == "eq":
            return f"{self.col} = {self.lo}"
        if self.kind == "range":
            return f"{self.col} BETWEEN {self.lo} AND {self.hi}"
        if self.kind == "in":
            return f"{self.col} IN ({', '.join(str(v) for v in self.values)})"
        if self.kind == "udf":
            return f"udf(price, qty, {UDF_MODULUS}) > {self.lo}"
        if self.kind == "or":
            return "(" + " OR ".join(p.text() for p in self.parts) + ")"
        raise ValueError(self.kind)


@dataclasses.dataclass
class Predicate:
    text: str
    terms: List[Term]
    target: float             # target selectivity
    est: float                # product of the terms' aimed selectivities
    seed: int


class _Rng:
    """Small scalar stream over the same counter-based generator (host-side)."""

    def __init__(self, seed: int, stream: int = 99):
        self.key = stream_key(seed, stream)
        self.i = 0

    def u64(self) -> int:
        self.i += 1
        return _mix_py((self.key + self.i * GAMMA) & MASK64)

    def uniform(self) -> float:
        return (self.u64() >> 11) * (2.0 ** -53)

    def randint(self, lo: int, hi: int) -> int:
        return lo + ((self.u64() >> 32) * (hi - lo + 1) >> 32)

    def choice(self, seq: Sequence):
        return seq[self.randint(0, len(seq) - 1)]

    def sample(self, lo: int, hi: int, k: int) -> List[int]:
        pool = list(range(lo, hi + 1))
        out = []
        for _ in range(k):
            j = self.randint(0, len(pool) - 1)
            out.append(pool.pop(j))
        return out


_ZIPF_KEY_CUM: Dict[Tuple[float, int, int], np.ndarray] = {}


def _zipf_key_cumulative(s: float, n: int, salt: int) -> np.ndarray:
    """cum[k] = P(key <= k) for the scattered Zipf keys (used to aim key ranges)."""
    k = (s, n, salt)
    if k not in _ZIPF_KEY_CUM:
        p = zipf_probabilities(s, n)
        keys = (np.arange(n, dtype=np.int64) * ZIPF_MULT + (salt % n)) % n
        by_key = np.empty(n, dtype=np.float64)
        by_key[keys] = p
        _ZIPF_KEY_CUM[k] = np.cumsum(by_key)
    return _ZIPF_KEY_CUM[k]


_KEY_SALT = {"key": 777, "key2": 4242}


def _range_term(rng: _Rng, col: str, s: float) -> Term:
    kind, lo, hi = SKEWED_SCHEMA[col]
    s = min(max(s, 0.0), 1.0)
    if kind == "zipf":
        cum = _zipf_key_cumulative(SKEWED_ZIPF_S, hi + 1, _KEY_SALT[col])
        a = rng.randint(lo, hi)
        base = cum[a - 1] if a > 0 else 0.0
        if base + s > 1.0:
            a = int(np.searchsorted(cum, max(0.0, 1.0 - s)))
            base = cum[a - 1] if a > 0 else 0.0
        b = int(min(np.searchsorted(cum, base + s), hi))
        return Term("range", col, a, b, est=float(cum[b] - base))
    d = hi - lo + 1
    width = max(1, min(d, int(round(s * d))))
    a = rng.randint(lo, hi - width + 1)
    return Term("range", col, a, a + width - 1, est=width / d)


def _eq_term(rng: _Rng, s: float, cands: Sequence[str]) -> Term:
    best = min(cands, key=lambda c: abs(math.log(max(s, 1e-12)) -
                                        math.log(1.0 / (SKEWED_SCHEMA[c][2] - SKEWED_SCHEMA[c][1] + 1))))
    _, lo, hi = SKEWED_SCHEMA[best]
    return Term("eq", best, rng.randint(lo, hi), est=1.0 / (hi - lo + 1))


def _in_term(rng: _Rng, s: float, cands: Sequence[str]) -> Term:
    col = rng.choice(cands)
    _, lo, hi = SKEWED_SCHEMA[col]
    k = hi - lo + 1
    n = max(2, min(16, k, int(round(s * k))))
    vals = tuple(sorted(rng.sample(lo, hi, n)))
    return Term("in", col, values=vals, est=n / k)


def _udf_term(rng: _Rng, s: float) -> Term:
    m = UDF_MODULUS
    k = int(round((m - 1) - s * m))
    k = max(-1, min(m - 1, k))
    return Term("udf", "price", lo=k, est=(m - 1 - k) / m)


def _or_term(rng: _Rng, s: float, cols: Sequence[str]) -> Term:
    part = 1.0 - math.sqrt(max(0.0, 1.0 - min(s, 1.0)))
    c1 = rng.choice(cols)
    c2 = rng.choice([c for c in cols if c != c1])
    a = _range_term(rng, c1, part)
    b = _range_term(rng, c2, part)
    if a.lo == a.hi:
        a = Term("eq", a.col, a.lo, est=a.est)
    return Term("or", parts=(a, b), est=a.est + b.est - a.est * b.est)


# Columns a term reads (a udf reads price and qty; an OR pair both of its columns).
def _term_columns(t: Term) -> Tuple[str, ...]:
    if t.kind == "udf":
        return ("price", "qty")
    if t.kind == "or":
        return tuple(c for p in t.parts for c in _term_columns(p))
    return (t.col,)


def random_predicate(seed: int, target: float, max_terms: int = 6) -> Predicate:
    """A conjunction of 1..max_terms terms aimed at selectivity `target`.

    The driver column (`price`, `day` or `key`; not `day` below a target of
    2e-3) is drawn first; the
    other terms are drawn on columns no earlier term reads, so that no two
    terms of the conjunction test the same column (two independent draws on
    one column are mostly disjoint, a contradiction that reads nothing).  The
    driver range is then sized so that the product of aimed selectivities
    equals the target.  Aims assume independent, uniform (or Zipf-known)
    columns; the achieved selectivity is whatever the exact count says (the
    correlated code columns make it differ).  A term kind whose columns are
    all taken, or whose coarse aim falls below the target, is replaced by a
    range on a free column, or dropped.
    """
    rng = _Rng(seed)
    nterms = rng.randint(1, max_terms)
    # `day` has 2,557 values: it cannot aim below 1/2557 alone
    driver_col = rng.choice(["price", "price", "day", "key"] if target >= 2e-3 else ["price", "price", "key"])
    used = {driver_col}
    others: List[Term] = []
    rem = math.log(target)      # log of the selectivity budget the terms drawn so far leave

    def free(cols):
        return [c for c in cols if c not in used]

    for _ in range(nterms - 1):
        kind = rng.choice(["eq", "range", "in", "or", "udf"])
        # spend a random share (up to half) of the remaining selectivity budget
        frac = rng.uniform() * 0.5
        s = math.exp(rem * frac) if rem < 0 else 1.0
        if kind == "eq" and free(["code7", "code25", "code150", "qty"]):
            t = _eq_term(rng, s, free(["code7", "code25", "code150", "qty"]))
        elif kind == "in" and free(["code25", "code150", "code7"]):
            t = _in_term(rng, s, free(["code25", "code150", "code7"]))
        elif kind == "or" and len(free(["day", "price", "qty", "code150", "key2"])) >= 2:
            t = _or_term(rng, s, free(["day", "price", "qty", "code150", "key2"]))
        elif kind == "udf" and not ({"price", "qty"} & used):
            t = _udf_term(rng, s)
        elif free(["day", "qty", "code150", "key", "key2"]):
            t = _range_term(rng, rng.choice(free(["day", "qty", "code150", "key", "key2"])), s)
        else:
            continue
        if t.est < math.exp(rem) and t.kind != "range":
            # a code test is coarse (1/7 of the rows at most for an equality):
            # where it would spend more than the whole remaining budget, a
            # range sized to the share takes its place
            if not free(["day", "qty", "code150", "key", "key2"]):
                continue
            t = _range_term(rng, rng.choice(free(["day", "qty", "code150", "key", "key2"])), s)
        used.update(_term_columns(t))
        others.append(t)
        rem = min(0.0, rem - math.log(max(t.est, 1e-300)))
    prod = 1.0
    for t in others:
        prod *= t.est
    driver_s = min(1.0, target / prod) if prod > 0 else 1.0
    driver = _range_term(rng, driver_col, driver_s)
    terms = [driver] + others
    order = list(range(len(terms)))
    for i in range(len(order) - 1, 0, -1):          # Fisher-Yates on the term order
        j = rng.randint(0, i)
        order[i], order[j] = order[j], order[i]
    terms = [terms[i] for i in order]
    est = 1.0
    for t in terms:
        est *= t.est
    return Predicate(" AND ".join(t.text() for t in terms), terms, target, est, seed)


def skewed_predicates(count: int = 200, seed0: int = 2000, lo_exp: float = -6.0,
                      hi_sel: float = 0.9) -> List[Predicate]:
    """`count` predicates with targets log-spaced from 10^lo_exp to hi_sel."""
    span = math.log10(hi_sel) - lo_exp
    out = []
    for j in range(count):
        t = 10.0 ** (lo_exp + span * j / max(1, count - 1))
        out.append(random_predicate(seed0 + j, t))
    return out


# ---------------------------------------------------------------- batched workload
BATCH_TABLE_ROWS = (10_000, 200_000, 2_000_000, 8_000_000, 30_000_000, 60_000_000)


def batch_workload(nqueries: int = 512, seed: int = 3,
                   sizes: Sequence[int] = BATCH_TABLE_ROWS) -> List[Tuple[int, Predicate]]:
    """(table index, predicate) pairs for the batched workload."""
    rng = _Rng(seed, stream=7)
    span = math.log10(0.9) + 6.0
    out = []
    for j in range(nqueries):
        ti = rng.randint(0, len(sizes) - 1)
        t = 10.0 ** (-6.0 + span * rng.uniform())
        out.append((ti, random_predicate(seed * 100_000 + j, t)))
    return out


# ---------------------------------------------------------------- star schema
STAR_DIM_ROWS = (2_000_000, 200_000, 30_000, 2_556)
STAR_ZIPF_S = 0.8


def star_fact(nrows: int = 600_000_000, seed: int = 4, device="cpu",
              dim_rows: Sequence[int] = STAR_DIM_ROWS) -> Table:
    """Fact table: fk0..fk3 Zipf(0.8) into dense dimension keys, m0, m1 measures."""
    cols = []
    for d, n in enumerate(dim_rows):
        cols.append(Column(f"fk{d}", "i32", _fill(nrows, "i32", device,
                    lambda s, c, d=d, n=n: zipf_keys(seed, d, s, c, STAR_ZIPF_S, n, device,
                                                     salt=1000 + 37 * d), chunk=1 << 26)))
    for m in range(2):
        cols.append(Column(f"m{m}", "i32", _fill(nrows, "i32", device,
                    lambda s, c, m=m: uniform_int(raw_u64(seed, 10 + m, s, c, device), 0, 100_000),
                    chunk=1 << 26)))
    return Table(nrows, cols)


def star_dim(d: int, nrows: int, seed: int = 4, device="cpu") -> Table:
    """Dimension table d: dense key = row index, attributes a (i32), b (i32), c (u8)."""
    base = 100 + 10 * d
    cols = [
        Column("a", "i32", _fill(nrows, "i32", device,
               lambda s, c: uniform_int(raw_u64(seed, base, s, c, device), 0, 999_999))),
        Column("b", "i32", _fill(nrows, "i32", device,
               lambda s, c: uniform_int(raw_u64(seed, base + 1, s, c, device), 0, 9_999))),
        Column("c", "u8", _fill(nrows, "u8", device,
               lambda s, c: uniform_int(raw_u64(seed, base + 2, s, c, device), 0, 24))),
    ]
    return Table(nrows, cols)


def star_dim_predicates(seed: int = 4, ndims: int = 4) -> List[str]:
    """One predicate per dimension, aimed at selectivities from 1e-3 to 0.5."""
    out = []
    for d in range(ndims):
        rng = _Rng(seed * 1000 + d, stream=5)
        target = 10.0 ** (-3.0 + (math.log10(0.5) + 3.0) * d / max(1, ndims - 1))
        width = max(1, int(round(target * 1_000_000)))
        lo = rng.randint(0, 1_000_000 - width)
        text = f"a BETWEEN {lo} AND {lo + width - 1}"
        if d % 2 == 1:
            text = f"({text} OR c = {rng.randint(0, 24)}) AND b < {rng.randint(5000, 9999)}"
        out.append(text)
    return out
