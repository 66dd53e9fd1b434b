"""Pins of the CPU oracle against things other than itself (no GPU).

* exhaustive brute force: a table holding every possible row over small
  domains, and a seeded sweep of predicates of up to 3 terms, checked against
  SQLite (an independent SQL engine) and the pure-Python evaluator;
* a hand-worked 10-row table (tests/golden/hand_worked.json);
* closed forms computed with numpy (bins, sorted searches, vectorised masks);
* invariants that hold at any size;
* SQLite on the full single table and on a sample of the skewed table with
  the headline workload's predicates.
"""
import itertools
import json
import os
import sqlite3

import numpy as np
import pytest

import oracle
from oracle import pyeval
from oracle.parse import parse, OracleParseError
from paper_1901_01488_gb300 import datagen

HERE = os.path.dirname(os.path.abspath(__file__))


def _sql(text: str) -> str:
    """Predicate text -> SQLite WHERE clause (udf(a, b, m) is (a * b) % m there)."""
    import re
    return re.sub(r"udf\(\s*(\w+)\s*,\s*(\w+)\s*,\s*(-?\d+)\s*\)", r"((\1 * \2) % \3)", text)


def _sqlite(cols, preds):
    con = sqlite3.connect(":memory:")
    names = list(cols)
    con.execute("CREATE TABLE t (id INTEGER PRIMARY KEY, " + ", ".join(f"{n} INTEGER" for n in names) + ")")
    n = len(next(iter(cols.values())))
    con.executemany(f"INSERT INTO t VALUES ({', '.join('?' * (len(names) + 1))})",
                    [(i, *[int(cols[c][i]) for c in names]) for i in range(n)])
    out = []
    for p in preds:
        out.append([r[0] for r in con.execute(f"SELECT id FROM t WHERE {_sql(p)} ORDER BY id")])
    con.close()
    return out


# ------------------------------------------------------------- brute force
def _all_rows_table():
    """Every row over a in {-2..3} (i32), b in {0..3} (u8), c in {-2..3} (i64)."""
    rows = list(itertools.product(range(-2, 4), range(0, 4), range(-2, 4)))
    a = np.array([r[0] for r in rows], dtype=np.int32)
    b = np.array([r[1] for r in rows], dtype=np.uint8)
    c = np.array([r[2] for r in rows], dtype=np.int64)
    return {"a": a, "b": b, "c": c}


def _atoms():
    out = []
    opds = ["a", "b", "c", "udf(a, c, 3)", "udf(b, a, 2)", "udf(c, c, 5)", "udf(a, b, 1)"]
    for o in opds:
        for op in ("=", "!=", "<", "<=", ">", ">="):
            for k in (-2, -1, 0, 1, 3, 4):
                out.append(f"{o} {op} {k}")
        for lo, hi in ((-1, 1), (0, 0), (2, 1), (-5, 5), (3, 9)):
            out.append(f"{o} BETWEEN {lo} AND {hi}")
            out.append(f"{o} NOT BETWEEN {lo} AND {hi}")
        for vals in ((), (0,), (1, 3), (-2, 0, 2), (3, 3, -1)):
            out.append(f"{o} IN ({', '.join(map(str, vals))})")
            out.append(f"{o} NOT IN ({', '.join(map(str, vals))})")
    out += ["TRUE", "FALSE"]
    return out


def _brute_preds(n=1500, seed=11):
    rng = np.random.default_rng(seed)
    atoms = _atoms()
    preds = list(atoms)
    shapes = ["{0} AND {1}", "{0} OR {1}", "NOT {0}", "NOT ({0} AND {1})", "{0} AND ({1} OR {2})",
              "({0} OR {1}) AND NOT {2}", "{0} OR {1} AND {2}", "NOT NOT {0}", "({0} OR {1} OR {2})"]
    for _ in range(n):
        s = shapes[rng.integers(len(shapes))]
        picks = [atoms[rng.integers(len(atoms))] for _ in range(3)]
        preds.append(s.format(*picks))
    return preds


def test_brute_force_vs_sqlite_and_python():
    cols = _all_rows_table()
    n = len(cols["a"])
    preds = _brute_preds()
    expect = _sqlite(cols, preds)
    for p, e in zip(preds, expect):
        ids, _ = oracle.select(p, cols)
        assert list(ids) == e, p
        assert oracle.count(p, cols) == len(e), p
        assert pyeval.select(parse(p), cols, n) == e, p


def test_parse_errors():
    for bad in ("", "a =", "a BETWEEN 1", "a IN (1,", "udf(a, b, 0) > 1", "a = 1 AND",
                "a NOT = 1", "a = 99999999999999999999", "(a = 1", "a = 1)", "a ? 1"):
        with pytest.raises(OracleParseError):
            parse(bad)


# ------------------------------------------------------------- hand-worked
def _hand():
    with open(os.path.join(HERE, "golden", "hand_worked.json")) as f:
        g = json.load(f)
    np_t = {"i32": np.int32, "i64": np.int64, "u8": np.uint8, "u16": np.uint16}
    cols = {k: np.array(v["values"], dtype=np_t[v["dtype"]]) for k, v in g["columns"].items()}
    return cols, g["cases"]


def test_hand_worked():
    cols, cases = _hand()
    for c in cases:
        ids, proj = oracle.select(c["predicate"], cols, ("key", "price"))
        assert list(ids) == c["ids"], c["predicate"]
        assert list(proj["key"]) == [cols["key"][i] for i in c["ids"]]
        assert oracle.count(c["predicate"], cols) == len(c["ids"])
        assert pyeval.select(parse(c["predicate"]), cols, 10) == c["ids"]
    # SQLite agrees with the hand-worked answers too
    got = _sqlite(cols, [c["predicate"] for c in cases])
    assert got == [c["ids"] for c in cases]


def _wrap_cases():
    with open(os.path.join(HERE, "golden", "hand_worked.json")) as f:
        return json.load(f)["wrap_cases"]


def test_hand_worked_udf_wraparound():
    """udf products that overflow 64 bits, worked by hand (golden file): the
    C oracle and the pure-Python evaluator both give the hand-worked ids."""
    cols, _ = _hand()
    for c in _wrap_cases():
        ids, _ = oracle.select(c["predicate"], cols)
        assert list(ids) == c["ids"], c["predicate"]
        assert oracle.count(c["predicate"], cols) == len(c["ids"]), c["predicate"]
        assert pyeval.select(parse(c["predicate"]), cols, 10) == c["ids"], c["predicate"]


_I64_EDGES = [-2**63, -2**63 + 1, -2**62, -2**32, -97, -1, 0, 1, 2, 96, 97,
              2**31 - 1, 2**32, 3037000500, 2**62, 2**63 - 1]


def test_udf_wraparound_sweep():
    """Every pair of 64-bit edge operands (256 rows) under moduli from 1 to
    2^63 - 1: the oracle's rows equal those of numpy's own wrapping uint64
    product and truncated int64 fmod, and those of the pure-Python evaluator
    (Python integers reduced mod 2^64).  Three independent evaluations of
    the udf reading (wrapping product, remainder truncated toward zero)."""
    pairs = [(x, y) for x in _I64_EDGES for y in _I64_EDGES]
    cols = {"x": np.array([p[0] for p in pairs], dtype=np.int64),
            "y": np.array([p[1] for p in pairs], dtype=np.int64)}
    n = len(pairs)
    prod = (cols["x"].view(np.uint64) * cols["y"].view(np.uint64)).view(np.int64)   # wraps mod 2^64
    for m in (1, 2, 97, 65535, 65536, 2**31 - 1, 2**32 + 15, 2**62 + 1, 2**63 - 1):
        r = np.fmod(prod, np.int64(m))                                             # sign of the dividend
        vals = sorted(set(r.tolist()))
        preds = [(f"udf(x, y, {m}) < 0", r < 0), (f"udf(x, y, {m}) > 0", r > 0),
                 (f"udf(y, x, {m}) = 0", r == 0)]
        for k in vals[:: max(1, len(vals) // 12)]:
            preds.append((f"udf(x, y, {m}) = {k}", r == k))
            preds.append((f"udf(x, y, {m}) BETWEEN {k} AND {min(k + 1000, 2**63 - 1)}", (r >= k) & (r <= k + 1000)))
            preds.append((f"udf(x, y, {m}) NOT IN ({k}, {-k if k != -2**63 else 0})",
                          ~((r == k) | (r == (-k if k != -2**63 else 0)))))
        for text, mask in preds:
            want = np.flatnonzero(mask).tolist()
            ids, _ = oracle.select(text, cols)
            assert ids.tolist() == want, text
            assert pyeval.select(parse(text), cols, n) == want, text


def test_u16_values_above_32767():
    """A u16 column holding values 32768..65535 is read zero-extended: the
    oracle agrees with SQLite (fed Python ints of the unsigned values), the
    pure-Python evaluator and numpy masks on the widened column."""
    dvals = [0, 1, 255, 256, 32767, 32768, 32769, 40000, 65534, 65535]
    avals = [-1, 0, 5]
    rows = [(d, a) for d in dvals for a in avals]
    cols = {"d": np.array([r[0] for r in rows], dtype=np.uint16),
            "a": np.array([r[1] for r in rows], dtype=np.int32)}
    n = len(rows)
    d = cols["d"].astype(np.int64)
    a = cols["a"].astype(np.int64)
    cases = [("d >= 32768", d >= 32768), ("d < 32768", d < 32768), ("d = 65535", d == 65535),
             ("d = -1", d == -1), ("d > -1", d > -1), ("d <= -32768", d <= -32768),
             ("d BETWEEN 32767 AND 32768", (d >= 32767) & (d <= 32768)),
             ("d BETWEEN -32768 AND 40000", d <= 40000),
             ("d IN (65535, -1, 32768, -32768)", (d == 65535) | (d == 32768)),
             ("d NOT IN (65534)", d != 65534),
             ("udf(d, d, 97) = 0", np.fmod(d * d, 97) == 0),
             ("udf(d, a, 1000003) < 0", np.fmod(d * a, 1000003) < 0),
             ("udf(a, d, 7) BETWEEN -6 AND -3", (np.fmod(a * d, 7) >= -6) & (np.fmod(a * d, 7) <= -3)),
             ("d > 40000 AND a = 5 OR d < 1", ((d > 40000) & (a == 5)) | (d < 1)),
             ("NOT (d BETWEEN 256 AND 65534)", (d < 256) | (d > 65534))]
    expect = _sqlite(cols, [c[0] for c in cases])
    for (text, mask), e in zip(cases, expect):
        want = np.flatnonzero(mask).tolist()
        assert e == want, text                     # SQLite agrees with the widened numpy mask
        ids, _ = oracle.select(text, cols)
        assert ids.tolist() == want, text
        assert pyeval.select(parse(text), cols, n) == want, text


# ------------------------------------------------------------- closed forms
@pytest.fixture(scope="module")
def single():
    return datagen.single_table(200_000, seed=1).host()


def test_equality_is_a_bincount_bin(single):
    bins = np.bincount(single["category"], minlength=25)
    for k in (0, 7, 24, 25, -1):
        assert oracle.count(f"category = {k}", single) == (bins[k] if 0 <= k < 25 else 0)


def test_between_is_a_sorted_search(single):
    s = np.sort(single["day"])
    for lo, hi in ((400, 765), (0, 2556), (2556, 2556), (10, 9), (-5, 3)):
        expect = max(0, np.searchsorted(s, hi, "right") - np.searchsorted(s, lo, "left"))
        assert oracle.count(f"day BETWEEN {lo} AND {hi}", single) == expect


def test_in_is_a_sum_of_bins(single):
    bins = np.bincount(single["category"], minlength=25)
    assert oracle.count("category IN (1, 3, 3, 24, 99)", single) == bins[1] + bins[3] + bins[24]


def test_vectorised_numpy_agrees(single):
    d = single
    m = (d["category"] == 7) & (d["day"] >= 400) & (d["day"] <= 765) & \
        ((d["price"] == 50000) | (d["price"] > 9_000_000))
    ids, proj = oracle.select(datagen.SINGLE_TABLE_PREDICATE, d, datagen.SINGLE_TABLE_PROJECTION)
    assert np.array_equal(ids, np.flatnonzero(m).astype(np.uint32))
    for p in datagen.SINGLE_TABLE_PROJECTION:
        assert np.array_equal(proj[p], d[p][ids])
    # udf with C (truncated) remainder: numpy fmod has the same sign rule
    u = np.fmod(d["price"] * d["day"].astype(np.int64), 97)
    assert oracle.count("udf(price, day, 97) > 40", d) == int(np.count_nonzero(u > 40))


def test_invariants(single):
    d = single
    n = len(d["day"])
    A = "day BETWEEN 100 AND 900"
    B = "category IN (2, 7, 11)"
    a, b = oracle.count(A, d), oracle.count(B, d)
    ab = oracle.count(f"{A} AND {B}", d)
    aob = oracle.count(f"{A} OR {B}", d)
    assert aob == a + b - ab
    assert ab <= min(a, b)
    assert oracle.count(f"NOT ({A})", d) == n - a
    prev = -1
    for w in (0, 10, 100, 1000, 2556):
        c = oracle.count(f"day BETWEEN 1000 AND {1000 + w}", d)
        assert c >= prev
        prev = c
    assert oracle.count(f"{A} AND price > 5000000", d) <= a
    ids, _ = oracle.select(f"{A} OR {B}", d)
    assert len(ids) == aob and np.all(np.diff(ids.astype(np.int64)) > 0)
    assert oracle.count_parallel(f"{A} OR {B}", d, 4) == aob


def test_single_table_statistical_sanity():
    """Not a pin: the 1M-row workload's count is near its expectation (572.6, sigma ~24)."""
    d = datagen.single_table(1_000_000, seed=1).host()
    c = oracle.count(datagen.SINGLE_TABLE_PREDICATE, d)
    assert abs(c - 572.6) < 6 * 24


@pytest.mark.slow
def test_single_table_vs_sqlite_full():
    d = datagen.single_table(1_000_000, seed=1).host()
    ids, _ = oracle.select(datagen.SINGLE_TABLE_PREDICATE, d)
    con = sqlite3.connect(":memory:")
    con.execute("CREATE TABLE t (id INTEGER PRIMARY KEY, key INTEGER, day INTEGER, price INTEGER, category INTEGER)")
    con.executemany("INSERT INTO t VALUES (?,?,?,?,?)",
                    zip(range(len(d["key"])), d["key"].tolist(), d["day"].tolist(),
                        d["price"].tolist(), d["category"].tolist()))
    got = [r[0] for r in con.execute(f"SELECT id FROM t WHERE {datagen.SINGLE_TABLE_PREDICATE} ORDER BY id")]
    assert got == ids.tolist()


# ------------------------------------------------------------- semi-join
def test_semijoin_pins():
    rng = np.random.default_rng(5)
    dims = (50, 7, 300)
    n = 20_000
    fk = [rng.integers(-2, D + 2, n).astype(np.int32) for D in dims]   # a few out-of-range keys
    marks = [(rng.random(D) < p).astype(np.uint8) for D, p in zip(dims, (0.3, 0.6, 0.05))]
    subsets = list(range(8))
    got = oracle.semijoin_counts(fk, marks, subsets)
    got4 = oracle.semijoin_counts(fk, marks, subsets, threads=4)
    assert got == got4
    assert got[0] == n
    # single dimension: sum over keys of mark * frequency (np.bincount)
    for d, D in enumerate(dims):
        f = fk[d]
        inr = (f >= 0) & (f < D)
        freq = np.bincount(f[inr], minlength=D)
        assert got[1 << d] == int(np.dot(freq, marks[d]))
    # any subset: vectorised boolean masks
    def ok(d):
        f = fk[d]
        inr = (f >= 0) & (f < dims[d])
        m = np.zeros(n, dtype=bool)
        m[inr] = marks[d][f[inr]] != 0
        return m
    for s in subsets:
        m = np.ones(n, dtype=bool)
        for d in range(3):
            if s >> d & 1:
                m &= ok(d)
        assert got[s] == int(m.sum())
    # monotone under subset inclusion
    for s in subsets:
        for t in subsets:
            if s & t == s:
                assert got[t] <= got[s]


def test_mark_matches_select():
    d = datagen.single_table(5_000, seed=9).host()
    p = "day < 1000 OR category = 3"
    m = oracle.mark(p, d)
    ids, _ = oracle.select(p, d)
    assert np.array_equal(np.flatnonzero(m), ids.astype(np.int64))


def test_skewed_sample_vs_sqlite():
    """The headline workload's 200 predicates on the first 200,000 rows of the
    skewed table: the oracle's counts equal SQLite's, and its ordered ids too
    (every fifth predicate)."""
    n = 200_000
    t = datagen.skewed_table(n)
    cols = t.host()
    texts = [p.text for p in datagen.skewed_predicates(200)]
    con = sqlite3.connect(":memory:")
    names = list(cols)
    con.execute("CREATE TABLE t (id INTEGER PRIMARY KEY, " + ", ".join(f"{c} INTEGER" for c in names) + ")")
    con.executemany(f"INSERT INTO t VALUES ({', '.join('?' * (len(names) + 1))})",
                    zip(range(n), *[cols[c].astype(np.int64).tolist() for c in names]))
    for j, text in enumerate(texts):
        want = con.execute(f"SELECT COUNT(*) FROM t WHERE {_sql(text)}").fetchone()[0]
        assert oracle.count(text, cols) == want, text
        if j % 5 == 0:
            ids = [r[0] for r in con.execute(f"SELECT id FROM t WHERE {_sql(text)} ORDER BY id")]
            got, _ = oracle.select(text, cols)
            assert got.tolist() == ids, text
    con.close()
