"""Host-side checks of libesc (no GPU): exports, compiler errors, the compiled
program's meaning (interpreted here with numpy, checked against the oracle),
and the udf divisor constants.  No kernel is launched."""
import os
import re

import numpy as np
import pytest
import torch

import oracle
from _helpers import host_table, as_columns, random_preds
from paper_1901_01488_gb300 import build as esc_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def esc():
    esc_build.build()
    from paper_1901_01488_gb300 import esc as m
    return m


def test_every_declared_symbol_is_exported(esc):
    with open(os.path.join(ROOT, "include", "esc.h")) as f:
        hdr = f.read()
    declared = set(re.findall(r"^\s*(?:esc_status|const char \*|uint64_t)\s*(esc_\w+)\s*\(", hdr, re.M))
    assert {"esc_table_create", "esc_predicate_compile", "esc_selectivity", "esc_selectivity_batch",
            "esc_semijoin_counts", "esc_bitmap_build"} <= declared
    for name in declared:
        assert hasattr(esc._lib, name), name
    assert declared <= set(esc.EXPORTED)


def _table(esc, cols):
    return esc.Table(as_columns(cols), len(next(iter(cols.values()))))


def _interpret(listing: str, cols):
    """Evaluates an EXPLAIN listing with numpy (this test's own interpreter)."""
    refs = {}
    stack = []
    n = None
    for line in listing.splitlines():
        f = line.split()
        if f[0] == "rows":
            n = int(f[1])
        elif f[0] == "ref":
            refs[int(f[1])] = cols[f[2]].astype(np.int64)
        elif f[0] == "instr":
            op = f[2]
            if op == "RANGE":
                x = refs[int(f[3])]
                stack.append((x >= int(f[5])) & (x <= int(f[6])))
            elif op == "IN":
                x = refs[int(f[3])]
                stack.append(np.isin(x, [int(v) for v in f[5].split(",")]))
            elif op == "UDF":
                a, b = refs[int(f[3])], refs[int(f[5])]
                with np.errstate(over="ignore"):
                    p = a * b
                r = np.fmod(p, int(f[7]))
                stack.append((r >= int(f[8])) & (r <= int(f[9])))
            elif op == "AND":
                y = stack.pop(); stack.append(stack.pop() & y)
            elif op == "OR":
                y = stack.pop(); stack.append(stack.pop() | y)
            elif op == "NOT":
                stack.append(~stack.pop())
            elif op in ("JZ", "JNZ"):
                pass  # skips work only when the result is already decided
            elif op == "TRUE":
                stack.append(np.ones(n, dtype=bool))
            elif op == "FALSE":
                stack.append(np.zeros(n, dtype=bool))
    assert len(stack) == 1
    return stack[0]


def test_compiled_program_means_the_predicate(esc):
    cols = host_table()
    t = _table(esc, cols)
    checked = 0
    for text in random_preds():
        try:
            p = esc.Predicate(t, text)
        except esc.EscError as e:
            assert "nests too deeply" in str(e) or "64 instructions" in str(e) or "pool" in str(e), (text, e)
            continue
        got = _interpret(p.explain(), cols)
        ids, _ = oracle.select(text, cols)
        assert np.array_equal(np.flatnonzero(got), ids.astype(np.int64)), text
        checked += 1
    assert checked > 300


def _same_operand_preds(count, seed):
    """Conjunctions and disjunctions of several tests on the same few operands
    (ranges, points, IN lists, udf both ways round), so that the compiler's
    merging of tests on one operand is exercised against the oracle."""
    rng = np.random.default_rng(seed)
    opds = ["a", "b", "udf(a, b, 7)", "udf(b, a, 7)", "udf(c, e, 97)", "udf(e, c, 97)"]

    def atom(o):
        k = rng.integers(5)
        v = int(rng.integers(-60, 60)) if o != "b" else int(rng.integers(-5, 260))
        if k == 0:
            return f"{o} {rng.choice(['=', '<', '<=', '>', '>='])} {v}"
        if k == 1:
            return f"{o} BETWEEN {v} AND {v + int(rng.integers(-3, 40))}"
        if k == 2:
            vals = ", ".join(str(v + int(rng.integers(-8, 8))) for _ in range(int(rng.integers(1, 6))))
            return f"{o} IN ({vals})"
        if k == 3:
            return f"{o} != {v}"
        return f"NOT ({o} BETWEEN {v} AND {v + 5})"

    out = []
    for _ in range(count):
        o = rng.choice(opds[:2] if rng.random() < 0.5 else opds)
        parts = [atom(o if rng.random() < 0.8 else rng.choice(opds)) for _ in range(int(rng.integers(2, 6)))]
        j = " AND " if rng.random() < 0.5 else " OR "
        inner = j.join(parts)
        out.append(inner if rng.random() < 0.7 else f"({inner}) {'OR' if j == ' AND ' else 'AND'} {atom(o)}")
    return out


def test_merged_tests_keep_the_meaning(esc):
    cols = host_table()
    t = _table(esc, cols)
    for text in _same_operand_preds(300, 5):
        got = _interpret(esc.Predicate(t, text).explain(), cols)
        ids, _ = oracle.select(text, cols)
        assert np.array_equal(np.flatnonzero(got), ids.astype(np.int64)), text


def test_tests_on_one_operand_merge(esc):
    t = _table(esc, host_table(100))

    def instrs(text):
        return [l.split(None, 2)[2] for l in esc.Predicate(t, text).explain().splitlines() if l.startswith("instr")]

    # AND intersects (udf operands in either order), OR unites adjacent ranges
    assert instrs("udf(c, a, 97) > 16 AND udf(a, c, 97) > 94") == ["UDF 0 i64 1 i32 97 95 96"]
    assert instrs("e = 3 AND e = 3") == ["RANGE 0 i32 3 3"]
    assert instrs("a BETWEEN 1 AND 5 OR a BETWEEN 6 AND 9 OR a = 20") == [
        "RANGE 0 i32 1 9", "RANGE 0 i32 20 20", "OR"]
    assert instrs("b IN (1, 4, 6) AND b BETWEEN 2 AND 9") == ["IN 0 u8 4,6"]
    assert instrs("a IN (1, 2, 3) OR a IN (3, 4)") == ["RANGE 0 i32 1 4"]          # one run: a range
    assert instrs("a IN (1, 2, 3) OR a IN (5, 6)") == ["IN 0 i32 1,2,3,5,6"]
    assert instrs("b IN (8, 5, 7, 6)") == ["RANGE 0 u8 5 8"]
    assert instrs("b IN (5, 7)") == ["IN 0 u8 5,7"]
    assert instrs("a IN (1, 2, 30) OR a BETWEEN 0 AND 10") == ["RANGE 0 i32 0 10", "RANGE 0 i32 30 30", "OR"]
    # empty conjunction, covering disjunction
    assert instrs("b = 1 AND b IN (4, 6)") == ["FALSE"]
    assert instrs("a = 2 AND (b = 1 AND b = 3)") == ["FALSE"]
    assert instrs("b < 100 OR b >= 50") == ["TRUE"]
    assert instrs("udf(b, d, 5) <= 2 OR udf(d, b, 5) > 1") == ["TRUE"]
    # different operands, or different moduli, stay apart
    assert [i.split()[0] for i in instrs("udf(c, a, 97) > 16 AND udf(c, a, 89) > 16")].count("UDF") == 2
    assert len(instrs("a = 1 AND e = 1")) == 3


def test_compile_errors(esc):
    cols = host_table(100)
    t = _table(esc, cols)
    bad = ["", "a =", "a BETWEEN 1", "a IN (1,", "udf(a, b, 0) > 1", "udf(a, b, -3) > 1",
           "zz = 1", "a = 1 AND", "a NOT = 1", "a = 99999999999999999999", "(a = 1", "a = 1)",
           "a ? 1", "a IN (" + ",".join(["1"] * 17) + ")"]
    for text in bad:
        with pytest.raises(esc.EscError) as ei:
            esc.Predicate(t, text)
        assert ei.value.status == esc.ESC_EINVAL, text
    with pytest.raises(esc.EscError):
        esc.Predicate(t, "a = 1", proj=("nope",))
    deep = "a = 1"
    for _ in range(10):
        deep = f"(b = 2 OR ({deep} AND c = 3))"
    p = esc.Predicate(t, deep)                      # Sethi-Ullman order keeps the stack shallow
    depth = int(p.explain().split("depth ")[1].split()[0])
    assert depth <= 3
    long = " AND ".join(f"a != {k}" for k in range(40))   # 40 tests + 39 ANDs > 64 instructions
    with pytest.raises(esc.EscError) as ei:
        esc.Predicate(t, long)
    assert "64 instructions" in str(ei.value)


def test_constant_folding_and_domains(esc):
    t = _table(esc, host_table(100))
    assert "FALSE" in esc.Predicate(t, "b > 255").explain()
    assert "TRUE" in esc.Predicate(t, "b >= 0").explain()
    assert "FALSE" in esc.Predicate(t, "d BETWEEN 70000 AND 80000").explain()
    assert "RANGE 0 i32 -2147483648 5" in esc.Predicate(t, "e <= 5").explain()
    assert "FALSE" in esc.Predicate(t, "a IN ()").explain()
    lst = esc.Predicate(t, "b IN (300, -1, 4, 4)").explain()
    assert "RANGE 0 u8 4 4" in lst
    assert "TRUE" in esc.Predicate(t, "NOT (b < 0)").explain()


def test_table_create_errors(esc):
    x = torch.zeros(64, dtype=torch.int32)
    with pytest.raises(esc.EscError):
        esc.esc_table_create([("a", "i32", x), ("a", "i32", x)], 64)
    with pytest.raises(esc.EscError) as ei:
        esc.esc_table_create([("a", "f32", x)], 64)
    assert ei.value.status == esc.ESC_ETYPE
    with pytest.raises(esc.EscError):
        esc.esc_table_create([("a", "i32", x[1:])], 63)       # not 16-byte aligned
    with pytest.raises(esc.EscError):
        esc.esc_table_create([("1a", "i32", x)], 64)
    with pytest.raises(esc.EscError):
        esc.esc_table_create([("a", "i32", x)], 1 << 32)
    with pytest.raises(esc.EscError) as ei:
        esc.esc_table_create([("a", "i32", x)], esc.MAX_ROWS + 1)    # an extent would pass 2^32
    assert ei.value.status == esc.ESC_EINVAL
    for n in (0, esc.MAX_ROWS):            # creating a table only records the pointers
        h = esc.esc_table_create([("a", "i32", x)], n)
        assert esc.esc_table_nrows(h) == n
        esc.esc_table_destroy(h)


def test_udf_magic_divides_exactly(esc):
    rng = np.random.default_rng(1)
    ds = [1, 2, 3, 7, 97, 1000, 1 << 20, (1 << 32) + 15, (1 << 62) + 1, (1 << 63) - 1, (1 << 63) + 5,
          (1 << 64) - 1] + [int(x) for x in rng.integers(1, 1 << 62, 40)]
    ns = [0, 1, (1 << 64) - 1, (1 << 63), (1 << 63) - 1] + [int(x) for x in rng.integers(0, 1 << 63, 200)]
    ns += [int(x) * 2 + 1 for x in rng.integers(0, 1 << 62, 50)]
    for d in ds:
        mult, s1, s2 = esc.esc_udf_magic(d)
        for n in ns + [d - 1, d, d + 1, 2 * d - 1, 2 * d]:
            n &= (1 << 64) - 1
            t = (mult * n) >> 64
            q = (t + ((n - t) >> s1)) >> s2
            assert q == n // d, (d, n)


def test_compile_many_matches_single_compiles(esc):
    """esc_predicate_compile_many: the same program as one compile per text
    (on several threads), and on a bad text every handle released and the
    lowest failing index named."""
    cols = host_table(4096, seed=9)
    t = _table(esc, cols)
    texts = [x for x in random_preds(600, seed=12)]
    good = []
    for x in texts:
        try:
            p = esc.Predicate(t, x, ("b", "c"))
            good.append((x, p.explain()))
            p.close()
        except esc.EscError:
            pass
    assert len(good) > 400
    for threads in (1, 3, 0):
        hs = esc.esc_predicate_compile_many(t.handle, [x for x, _ in good], ("b", "c"), threads)
        assert [esc.esc_predicate_explain(h) for h in hs] == [e for _, e in good]
        for h in hs:
            esc.esc_predicate_destroy(h)
    bad = [x for x, _ in good[:300]]
    bad[170] = "b < "
    bad[250] = "nosuchcolumn = 1"
    with pytest.raises(esc.EscError, match="predicate 170"):
        esc.esc_predicate_compile_many(t.handle, bad, (), 4)
    assert esc.esc_predicate_compile_many(t.handle, [], ()) == []
    ps = esc.PredicateSet(t, ["a < 3", "b IN (1, 2)"], ("a",))
    assert len(ps) == 2 and all(ps.handles)
    ps.close()


def test_headline_predicates_read_columns(esc):
    """Every one of the 200 headline predicates compiles to a program that
    reads at least one column: none folds to a constant TRUE or FALSE."""
    from paper_1901_01488_gb300 import datagen
    t = datagen.skewed_table(4096)
    tbl = esc.Table.from_datagen(t)
    for p in datagen.skewed_predicates(200):
        listing = esc.Predicate(tbl, p.text, datagen.SKEWED_PROJECTION).explain()
        assert any(l.startswith("ref ") for l in listing.splitlines()), p.text


def test_checked_build_loads_and_says_so(esc):
    """The checked build (kernels that test their indices) exports the same
    symbols and reports itself as checked; the release build does not."""
    import subprocess
    import sys
    assert esc.esc_build_checked() is False
    code = ("import sys; sys.path.insert(0, sys.argv[1]); from paper_1901_01488_gb300 import esc; "
            "assert esc.LIB_PATH.endswith('libesc_checked.so'); assert esc.esc_build_checked() is True; "
            "[getattr(esc._lib, n) for n in esc.EXPORTED]; print('ok')")
    env = dict(os.environ, ESC_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr


def test_write_unit_layout(esc):
    """Compaction units of a materialising call: 1..256 groups of 256 rows
    each, covering every group; with `slots` write-kernel blocks resident,
    as many whole waves as 256-group units need, with units as small as
    fill them; a batch (slots 0) keeps 256-group units.  The group-to-unit
    reciprocal divides every group index of the largest table exactly."""
    rng = np.random.default_rng(5)
    sizes = [0, 1, 255, 256, 257, 65536, 65537, 1_000_000, 8_000_000, 39_845_888, 39_845_889,
             60_000_000, 600_000_000, esc.MAX_ROWS] + [int(x) for x in rng.integers(1, esc.MAX_ROWS, 30)]
    for slots in (0, 1, 7, 608, 1216):
        for n in sizes:
            ug, nw, _ = esc.esc_debug_write_units(n, slots)
            groups = (n + 255) // 256
            assert 1 <= ug <= 256, (n, slots, ug)
            assert nw == -(-groups // ug), (n, slots)
            if slots == 0:
                assert ug == 256
            elif groups:
                waves = -(-groups // (256 * slots))
                assert -(-nw // slots) == waves, (n, slots, nw)
                if ug > 1:   # one group fewer per unit would need another wave
                    assert -(-groups // (ug - 1)) > waves * slots, (n, slots, ug)
    top = (esc.MAX_ROWS + 255) // 256          # group indices run below this
    for ug in range(1, 257):
        got, nw, recip = esc.esc_debug_write_units(256 * ug, 1)
        assert (got, nw) == (ug, 1)
        gs = {0, 1, ug - 1, ug, ug + 1, top - 1, top - 2} | {k * ug + d for k in (top // ug - 1, top // ug)
                                                              for d in (-1, 0, 1)}
        gs |= {int(x) for x in rng.integers(0, top, 200)}
        for g in sorted(x for x in gs if 0 <= x < top):
            assert ((g * recip) >> 32 if recip else g) == g // ug, (ug, g)
    with pytest.raises(esc.EscError):
        esc.esc_debug_write_units(esc.MAX_ROWS + 1, 608)
    with pytest.raises(esc.EscError):
        esc.esc_debug_write_units(1000, -1)
