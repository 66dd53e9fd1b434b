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
