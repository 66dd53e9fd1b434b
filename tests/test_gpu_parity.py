"""GPU parity: every count and row list from the CUDA path equals the oracle's,
bit for bit, on the same seeded inputs (all through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
from _helpers import host_table, as_columns, random_preds
from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def esc():
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc as m
    return m


def _check(esc, host, table, text, proj=(), capacity=None):
    """Count + ordered rows + projected values equal the oracle's."""
    p = esc.Predicate(table, text, proj)
    exp_ids, exp_proj = oracle.select(text, host, proj)
    n = esc.count(table, p)
    assert n == len(exp_ids), text
    cnt, ids, cols = esc.select(table, p, capacity=capacity)
    assert cnt == len(exp_ids), text
    got = ids.cpu().numpy().view(np.uint32)
    k = len(got)
    assert np.array_equal(got, exp_ids[:k]), text
    for name, c in zip(proj, cols):
        g = c.cpu().numpy()
        if host[name].dtype == np.uint16:
            g = g.view(np.uint16)
        assert np.array_equal(g, exp_proj[name][:k]), (text, name)
    return n


def test_single_table_full(esc):
    t = datagen.single_table(1_000_000, seed=1, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    n = _check(esc, host, tbl, datagen.SINGLE_TABLE_PREDICATE, datagen.SINGLE_TABLE_PROJECTION)
    assert 400 < n < 750


SIZES = [0, 1, 2, 15, 16, 17, 31, 32, 33, 255, 256, 257, 511, 512, 513, 2047, 2048, 2049,
         4097, 8191, 65537, 100_003]
TAIL_PREDS = ["day < 1500", "category IN (1, 2, 3) OR price > 5000000", "TRUE", "FALSE",
              datagen.SINGLE_TABLE_PREDICATE, "udf(price, day, 97) > 40", "category = 3",
              "NOT (key BETWEEN 1000 AND 900000) AND category != 4"]


@pytest.mark.parametrize("n", SIZES)
def test_tail_sizes(esc, n):
    t = datagen.single_table(n, seed=5, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    for text in TAIL_PREDS:
        _check(esc, host, tbl, text, ("key", "day", "price", "category"))


def test_random_predicates_all_types(esc):
    host = host_table(300_001, seed=21)
    tbl = esc.Table(as_columns(host, "cuda"), 300_001)
    done = 0
    for text in random_preds(160, seed=5):
        try:
            _check(esc, host, tbl, text, ("b", "c", "d", "e"))
            done += 1
        except esc.EscError as e:
            assert "64 instructions" in str(e) or "pool" in str(e), (text, e)
    assert done > 120


def test_in_set_forms(esc):
    """IN lists: the 256-bit set of values 0..255 and the general list, on
    every column type (negative and out-of-range column values included):
    word boundaries of the set (31/32, 63/64, 255), negative and repeated
    values, negation, and use inside AND/OR."""
    host = host_table(100_003, seed=31)
    tbl = esc.Table(as_columns(host, "cuda"), 100_003)
    lists = ["0", "31", "32", "63", "64", "0, 3, 31", "1, 33, 63", "32, 40, 47", "0, 31, 32, 63",
             "5, 64, 200", "63, 64", "255", "0, 255", "-1, 0, 1, 31", "2, 2, 2"]
    n = 0
    for col in ("a", "b", "c", "d", "e"):
        for lst in lists:
            for text in (f"{col} IN ({lst})", f"NOT {col} IN ({lst})",
                         f"({col} IN ({lst}) OR a = 7) AND b IN ({lst})"):
                n += _check(esc, host, tbl, text, ("a", "b"))
    assert n > 0


def test_truncation(esc):
    t = datagen.single_table(50_000, seed=7, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    text = "day < 2000"
    p = esc.Predicate(tbl, text, ("price",))
    exp_ids, exp_proj = oracle.select(text, host, ("price",))
    rows = p.alloc_rows(100)
    cnt, st = esc.esc_selectivity(tbl.handle, p.handle, rows)
    assert st == esc.ESC_ETRUNC and cnt == len(exp_ids)
    assert np.array_equal(rows[1].cpu().numpy().view(np.uint32)[:100], exp_ids[:100])
    assert np.array_equal(rows[2][0].cpu().numpy()[:100], exp_proj["price"][:100])
    cnt0, st0 = esc.esc_selectivity(tbl.handle, p.handle, (0, None, []))
    assert st0 == esc.ESC_ETRUNC and cnt0 == len(exp_ids)


def test_constant_programs(esc):
    """Predicates that fold to TRUE or FALSE (no column read) take no scan:
    counts, rows, truncation, bitmaps and the allocation-free entry point."""
    n = 5_003
    cols = host_table(n, seed=9)
    tbl = esc.Table(as_columns(cols, "cuda"), n)
    cases = [("TRUE", n), ("FALSE", 0), ("b = 1 AND b = 2", 0), ("b < 100 OR b >= 50", n),
             ("NOT (a = 1 AND a = 2)", n), ("udf(c, a, 7) > 6", 0), ("d BETWEEN 70000 AND 80000 OR TRUE", n)]
    for text, exp in cases:
        p = esc.Predicate(tbl, text, ("c", "b"))
        assert not any(l.startswith("ref ") for l in p.explain().splitlines()), text
        assert esc.count(tbl, p) == exp == oracle.count(text, cols), text
        ids_o, proj_o = oracle.select(text, cols, ("c", "b"))
        cnt, ids, proj = esc.select(tbl, p)
        assert cnt == exp and np.array_equal(ids.cpu().numpy().view(np.uint32), ids_o), text
        assert np.array_equal(proj[0].cpu().numpy(), proj_o["c"]) and np.array_equal(proj[1].cpu().numpy(), proj_o["b"])
        rows = p.alloc_rows(100)
        c2, st = esc.esc_selectivity(tbl.handle, p.handle, rows)
        assert c2 == exp and st == (esc.ESC_ETRUNC if exp > 100 else esc.ESC_OK)
        assert np.array_equal(rows[1].cpu().numpy().view(np.uint32)[:min(exp, 100)], ids_o[:100])
        c3, _ = esc.esc_selectivity_noalloc(tbl.handle, p.handle, p.alloc_rows(n))
        assert c3 == exp
        bm = torch.full(((n + 31) // 32,), -1, dtype=torch.int32, device="cuda")
        assert esc.esc_bitmap_build(tbl.handle, p.handle, bm) == exp
        bits = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")
        assert bits[:n].sum() == exp and bits[n:].sum() == 0, text     # tail bits clear


def test_skewed_table_2m(esc):
    t = datagen.skewed_table(2_000_000, seed=2, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    preds = datagen.skewed_predicates(200)
    for p in preds[::5]:
        _check(esc, host, tbl, p.text, datagen.SKEWED_PROJECTION)


def test_skewed_full_size(esc):
    """The 60M-row workload as the benchmark times it, checked in full for a few predicates."""
    t = datagen.skewed_table(60_000_000, seed=2, device="cuda")
    # generator is device-independent: spot-check rows against a CPU regeneration
    cpu = datagen.skewed_table(200_000, seed=2, device="cpu")
    for c_gpu, c_cpu in zip(t.columns, cpu.columns):
        assert torch.equal(c_gpu.data[:200_000].cpu(), c_cpu.data)
    tbl = esc.Table.from_datagen(t)
    preds = datagen.skewed_predicates(200)
    for j in (0, 90, 199):
        text = preds[j].text
        cols = oracle.columns_of(oracle.parse(text))
        need = list(dict.fromkeys(cols + list(datagen.SKEWED_PROJECTION)))
        host = {c: t.col(c).numpy() for c in need}
        _check(esc, host, tbl, text, datagen.SKEWED_PROJECTION)


def test_skewed_full_size_every_predicate(esc):
    """All 200 predicates of the benchmark at 60M rows, in select mode as it
    runs them: properties that hold at any size (count = count-mode count,
    ids strictly increasing and in range, projected values = the table's
    values at those ids), and 64 sampled rows per predicate decided by the
    oracle one by one (a 64-row table of those rows) against membership in
    the returned ids."""
    t = datagen.skewed_table(60_000_000, seed=2, device="cuda")
    tbl = esc.Table.from_datagen(t)
    proj = datagen.SKEWED_PROJECTION
    rng = np.random.default_rng(11)
    for j, pd in enumerate(datagen.skewed_predicates(200)):
        p = esc.Predicate(tbl, pd.text, proj)
        n_count = esc.count(tbl, p)
        n, ids, cols = esc.select(tbl, p, capacity=n_count)
        assert n == n_count == ids.numel(), j
        ids64 = ids.to(torch.int64) & 0xffffffff
        if n:
            assert int(ids64[0]) >= 0 and int(ids64[-1]) < t.nrows
            assert bool((ids64[1:] > ids64[:-1]).all()), j
            for name, c in zip(proj, cols):
                assert torch.equal(c, t.col(name).data.index_select(0, ids64)), (j, name)
        sample = np.sort(rng.choice(t.nrows, 64, replace=False))
        sidx = torch.from_numpy(sample).cuda()
        host = {c.name: c.data.index_select(0, sidx).cpu().numpy() for c in t.columns}
        for c in t.columns:
            if c.dtype == "u16":
                host[c.name] = host[c.name].view(np.uint16)
        want = np.zeros(64, dtype=bool)
        want[oracle.select(pd.text, host)[0].astype(np.int64)] = True
        got = torch.isin(sidx, ids64).cpu().numpy()
        assert np.array_equal(got, want), (j, pd.text)


def test_async_and_two_streams(esc):
    t = datagen.single_table(3_000_000, seed=8, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    texts = ["day BETWEEN 10 AND 1000", "category IN (3, 4) AND price < 600000"]
    exp = [oracle.count(x, host) for x in texts]
    preds = [esc.Predicate(tbl, x) for x in texts]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    for _ in range(3):
        esc.esc_selectivity_async(tbl.handle, preds[0].handle, out[0:1], None, s1)
        esc.esc_selectivity_async(tbl.handle, preds[1].handle, out[1:2], None, s2)
        torch.cuda.synchronize()
        assert out.tolist() == exp


def test_batch_matches_single(esc):
    tabs = [datagen.skewed_table(n, seed=30 + i, device="cuda") for i, n in enumerate((10_000, 200_000, 2_000_001))]
    etabs = [esc.Table.from_datagen(t) for t in tabs]
    hosts = [t.host() for t in tabs]
    work = datagen.batch_workload(48, seed=3, sizes=(10_000, 200_000, 2_000_001))
    preds, rows, expect = [], [], []
    for j, (ti, p) in enumerate(work):
        pr = esc.Predicate(etabs[ti], p.text, datagen.SKEWED_PROJECTION)
        preds.append(pr)
        ids, proj = oracle.select(p.text, hosts[ti], datagen.SKEWED_PROJECTION)
        expect.append((ids, proj))
        rows.append(pr.alloc_rows(len(ids) + 3) if j % 3 else None)   # every third is count-only
    counts, st = esc.esc_selectivity_batch([etabs[ti].handle for ti, _ in work], [p.handle for p in preds], rows)
    assert st == esc.ESC_OK
    for j in range(len(work)):
        ids, proj = expect[j]
        assert counts[j] == len(ids)
        if rows[j] is not None:
            got = rows[j][1][:len(ids)].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ids)
            for name, c in zip(datagen.SKEWED_PROJECTION, rows[j][2]):
                assert np.array_equal(c[:len(ids)].cpu().numpy(), proj[name])
    # prepared batch replayed from its CUDA graph, twice
    b = esc.esc_batch_prepare([etabs[ti].handle for ti, _ in work], [p.handle for p in preds], rows)
    dev_counts = torch.zeros(len(work), dtype=torch.int64, device="cuda")
    done = torch.zeros(len(work), dtype=torch.int64, device="cuda")
    for _ in range(2):
        dev_counts.zero_()
        esc.esc_batch_run(b, dev_counts, done)
        torch.cuda.synchronize()
        assert dev_counts.tolist() == counts
        assert bool((done > 0).all())
    esc.esc_batch_destroy(b)


def test_batch_with_constant_programs(esc):
    """Batches mixing constant programs (no work units; the constant kernel
    answers them, TRUE with every row) with scanned ones: counts, rows and
    completion times, prepared, one-shot and asynchronous."""
    t = datagen.skewed_table(300_007, seed=31, device="cuda")
    tbl = esc.Table.from_datagen(t)
    host = t.host()
    proj = datagen.SKEWED_PROJECTION
    texts = ["FALSE", "day < 100", "code7 = 1 AND code7 = 2", "TRUE", "price > 9000000",
             "qty < 5 OR qty >= 5", "key IN (1, 2, 3) AND key = 9", "day BETWEEN 5 AND 9"]
    preds = [esc.Predicate(tbl, x, proj) for x in texts]
    expect = [oracle.select(x, host, proj) for x in texts]
    rows = [p.alloc_rows(len(e[0]) + 1) if j % 2 == 0 else None for j, (p, e) in enumerate(zip(preds, expect))]
    counts, st = esc.esc_selectivity_batch([tbl.handle] * len(texts), [p.handle for p in preds], rows)
    assert st == esc.ESC_OK and counts == [len(e[0]) for e in expect]
    for r, (ids, pv) in zip(rows, expect):
        if r is not None:
            assert np.array_equal(r[1][:len(ids)].cpu().numpy().view(np.uint32), ids)
            for name, c in zip(proj, r[2]):
                assert np.array_equal(c[:len(ids)].cpu().numpy(), pv[name])
    b = esc.esc_batch_prepare([tbl.handle] * len(texts), [p.handle for p in preds], rows)
    dev_counts = torch.zeros(len(texts), dtype=torch.int64, device="cuda")
    done = torch.zeros(len(texts), dtype=torch.int64, device="cuda")
    esc.esc_batch_run(b, dev_counts, done)
    torch.cuda.synchronize()
    assert dev_counts.tolist() == counts and bool((done > 0).all())
    esc.esc_batch_destroy(b)
    dev_counts.zero_()
    done.zero_()
    esc.esc_selectivity_batch_async([tbl.handle] * len(texts), [p.handle for p in preds], dev_counts, rows, done)
    torch.cuda.synchronize()
    assert dev_counts.tolist() == counts and bool((done > 0).all())
    # all constant: nothing to scan at all
    consts = [preds[0], preds[2], preds[3]]
    c2, _ = esc.esc_selectivity_batch([tbl.handle] * 3, [p.handle for p in consts])
    assert c2 == [0, 0, t.nrows]


def test_shared_scan(esc):
    """Counts of many predicates in one pass (shared scan) equal the oracle's:
    random predicates over every type on a ragged table, passes split by the
    16 stage slots (a 20-column table), more than 2048 predicates, an empty
    table."""
    n = 100_003
    cols = host_table(n, seed=13)
    t = esc.Table(as_columns(cols, "cuda"), n)
    texts, preds = [], []
    for x in random_preds(300, seed=23):
        try:
            preds.append(esc.Predicate(t, x))
            texts.append(x)
        except esc.EscError:
            pass
    dev = torch.zeros(len(preds), dtype=torch.int64, device="cuda")
    esc.esc_selectivity_shared_async(t.handle, [p.handle for p in preds], dev)
    assert dev.tolist() == [oracle.count(x, cols) for x in texts]
    # 20 columns: one predicate per column pair, so the union exceeds 16 slots
    rng = np.random.default_rng(3)
    wide = {f"x{k}": rng.integers(-1000, 1000, 50_001).astype(np.int32) for k in range(20)}
    tw = esc.Table(as_columns(wide, "cuda"), 50_001)
    wtexts = [f"x{k} > {int(rng.integers(-900, 900))} AND x{(k + 7) % 20} < {int(rng.integers(-900, 900))}"
              for k in range(20)] * 3
    wp = [esc.Predicate(tw, x) for x in wtexts]
    dev = torch.zeros(len(wp), dtype=torch.int64, device="cuda")
    esc.esc_selectivity_shared_async(tw.handle, [p.handle for p in wp], dev)
    assert dev.tolist() == [oracle.count(x, wide) for x in wtexts]
    # more than one pass of 2048 predicates
    many = [preds[k % len(preds)] for k in range(2100)]
    dev = torch.zeros(len(many), dtype=torch.int64, device="cuda")
    esc.esc_selectivity_shared_async(t.handle, [p.handle for p in many], dev)
    single = [esc.count(t, p) for p in preds]
    assert dev.tolist() == [single[k % len(preds)] for k in range(2100)]
    # an empty table
    t0 = esc.Table(as_columns({k: v[:0] for k, v in cols.items()}, "cuda"), 0)
    p0 = [esc.Predicate(t0, "a > 1"), esc.Predicate(t0, "TRUE")]
    dev = torch.full((2,), 7, dtype=torch.int64, device="cuda")
    esc.esc_selectivity_shared_async(t0.handle, [p.handle for p in p0], dev)
    assert dev.tolist() == [0, 0]


def test_bitmap_and_semijoin(esc):
    dims_rows = datagen.STAR_DIM_ROWS
    fact = datagen.star_fact(3_000_017, seed=4, device="cuda", dim_rows=dims_rows)
    ftab = esc.Table.from_datagen(fact)
    texts = datagen.star_dim_predicates(4)
    bitmaps, marks = [], []
    for d, nrows in enumerate(dims_rows):
        dim = datagen.star_dim(d, nrows, seed=4, device="cuda")
        dtab = esc.Table.from_datagen(dim)
        p = esc.Predicate(dtab, texts[d])
        bm = torch.zeros((nrows + 31) // 32, dtype=torch.int32, device="cuda")
        cnt = esc.esc_bitmap_build(dtab.handle, p.handle, bm)
        mk = oracle.mark(texts[d], dim.host())
        bits = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")[:nrows]
        assert np.array_equal(bits, mk), d
        assert cnt == int(mk.sum())
        bitmaps.append(bm)
        marks.append(mk)
    fk = [fact.col(f"fk{d}").numpy() for d in range(4)]
    got = esc.esc_semijoin_counts(ftab.handle, [f"fk{d}" for d in range(4)], bitmaps, list(dims_rows))
    exp = oracle.semijoin_counts(fk, marks, list(range(16)), threads=8)
    assert got == [exp[s] for s in range(16)]
    # fewer dimensions, and foreign keys outside the dimension (not matches)
    got2 = esc.esc_semijoin_counts(ftab.handle, ["fk3", "fk1"], [bitmaps[3], bitmaps[1]],
                                   [dims_rows[3] - 100, dims_rows[1]])
    m3 = marks[3].copy()
    m3 = m3[:dims_rows[3] - 100]
    exp2 = oracle.semijoin_counts([fk[3], fk[1]], [m3, marks[1]], [0, 1, 2, 3])
    assert got2 == [exp2[s] for s in range(4)]


@pytest.mark.parametrize("dims_rows", [[0, 37, 1_000_000, 70], [9_000_000, 37, 1_000_000, 70]])
def test_semijoin_edges(esc, dims_rows):
    """Keys outside [0, rows) (negative, past the end, the int32 extremes), a
    dimension with no rows, one or two too large for shared memory (probed in
    place: 1M rows, and 9M rows beside it), and bitmaps whose bits past the
    last row are set."""
    rng = np.random.default_rng(8)
    n = 200_003
    fk, marks, bms = [], [], []
    for d, rows in enumerate(dims_rows):
        k = rng.integers(-40, rows + 40, n).astype(np.int32)
        k[rng.integers(0, n, 50)] = np.iinfo(np.int32).min
        k[rng.integers(0, n, 50)] = np.iinfo(np.int32).max
        fk.append(k)
        words = (rows + 31) // 32
        w = rng.integers(0, 2**32, max(words, 1), dtype=np.uint64).astype(np.uint32)  # garbage past `rows` too
        bits = np.unpackbits(w.view(np.uint8), bitorder="little")[:rows]
        marks.append(bits.astype(np.uint8))
        bms.append(torch.from_numpy(w.view(np.int32).copy()).cuda() if words else None)
    cols = [(f"fk{d}", "i32", torch.from_numpy(fk[d]).cuda()) for d in range(4)]
    tbl = esc.Table(cols, n)
    for sel in ([0, 1, 2, 3], [2, 0], [3], [1, 2]):
        got = esc.esc_semijoin_counts(tbl.handle, [f"fk{d}" for d in sel], [bms[d] for d in sel],
                                      [dims_rows[d] for d in sel])
        exp = oracle.semijoin_counts([fk[d] for d in sel], [marks[d] for d in sel], list(range(1 << len(sel))))
        assert got == [exp[s] for s in range(1 << len(sel))], sel


def test_empty_table(esc):
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    tbl = esc.Table([("a", "i32", x)], 0)
    p = esc.Predicate(tbl, "a = 0", ("a",))
    assert esc.count(tbl, p) == 0
    n, ids, cols = esc.select(tbl, p, capacity=4)
    assert n == 0 and len(ids) == 0


def test_bounded_wait_reports_timeout(esc):
    st = esc.esc_selftest_wait_timeout(200_000_000)
    assert st == esc.ESC_ETIMEOUT
    # the context is still usable
    t = datagen.single_table(10_000, seed=1, device="cuda")
    tbl = esc.Table.from_datagen(t)
    p = esc.Predicate(tbl, "day < 100")
    assert esc.count(tbl, p) == oracle.count("day < 100", t.host())


def test_hand_worked_golden_cases(esc):
    """The hand-worked golden table (tests/golden/hand_worked.json), its plain
    cases and its udf products that overflow 64 bits, through the C ABI: ids
    and projected values equal the hand-worked ids (no oracle involved)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_worked.json")) as f:
        g = json.load(f)
    np_t = {"i32": np.int32, "i64": np.int64, "u8": np.uint8, "u16": np.uint16}
    host = {k: np.array(v["values"], dtype=np_t[v["dtype"]]) for k, v in g["columns"].items()}
    tbl = esc.Table(as_columns(host, "cuda"), 10)
    for c in g["cases"] + g["wrap_cases"]:
        p = esc.Predicate(tbl, c["predicate"], ("key", "big"))
        n, ids, cols = esc.select(tbl, p)
        assert n == len(c["ids"]) and esc.count(tbl, p) == n, c["predicate"]
        assert ids.cpu().numpy().view(np.uint32).tolist() == c["ids"], c["predicate"]
        assert cols[0].cpu().numpy().tolist() == [int(host["key"][i]) for i in c["ids"]]
        assert cols[1].cpu().numpy().tolist() == [int(host["big"][i]) for i in c["ids"]]


def test_batch_in_waves_matches_oracle(esc):
    """A batch prepared in waves (smallest sub-queries first, work doubling
    per wave): counts, ordered ids and projected values equal the oracle's,
    replayed twice from its CUDA graph, and the sub-queries of the smallest
    tables complete earlier than those of the largest (medians)."""
    sizes = (10_000, 200_000, 2_000_001)
    tabs = [datagen.skewed_table(n, seed=40 + i, device="cuda") for i, n in enumerate(sizes)]
    etabs = [esc.Table.from_datagen(t) for t in tabs]
    hosts = [t.host() for t in tabs]
    work = datagen.batch_workload(60, seed=4, sizes=sizes)
    proj = datagen.SKEWED_PROJECTION
    preds, rows, expect = [], [], []
    for j, (ti, p) in enumerate(work):
        pr = esc.Predicate(etabs[ti], p.text, proj)
        preds.append(pr)
        ids, pv = oracle.select(p.text, hosts[ti], proj)
        expect.append((ids, pv))
        rows.append(pr.alloc_rows(len(ids) + 2) if j % 3 else None)   # every third count-only
    b = esc.esc_batch_prepare_waves([etabs[ti].handle for ti, _ in work], [p.handle for p in preds], rows, waves=4)
    dc = torch.zeros(len(work), dtype=torch.int64, device="cuda")
    done = torch.zeros(len(work), dtype=torch.int64, device="cuda")
    t0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        for r in rows:
            if r is not None:
                r[1].fill_(-1)
        dc.zero_()
        esc.esc_timestamp(t0)
        esc.esc_batch_run(b, dc, done)
        torch.cuda.synchronize()
        counts = dc.tolist()
        for j, (ids, pv) in enumerate(expect):
            assert counts[j] == len(ids), work[j][1].text
            if rows[j] is not None:
                assert np.array_equal(rows[j][1][:len(ids)].cpu().numpy().view(np.uint32), ids), work[j][1].text
                for name, c in zip(proj, rows[j][2]):
                    assert np.array_equal(c[:len(ids)].cpu().numpy(), pv[name]), (work[j][1].text, name)
        lat = (done - t0).tolist()
        assert all(x > 0 for x in lat)
        small = [lat[j] for j, (ti, _) in enumerate(work) if ti == 0]
        large = [lat[j] for j, (ti, _) in enumerate(work) if ti == 2]
        assert np.median(small) < np.median(large), (np.median(small), np.median(large))
    esc.esc_batch_destroy(b)
    with pytest.raises(esc.EscError):
        esc.esc_batch_prepare_waves([etabs[0].handle], [preds[0].handle], None, waves=0)
