"""A table of the most rows a table may hold (2^32 - 2^16 rows of one u8
column, 4.29 GB): counts, ordered ids near the top of the uint32 row-id
range, the dense-key bitmap, the shared scan, a batch and the allocation-free
call, against closed forms over the whole table and against the oracle on
its last 2^20 rows.

Column a holds row mod 251, so the rows with a = v are v, v + 251, ...: the
count of `a = v` over n rows is (n - 1 - v) // 251 + 1, and range and set
counts are sums of those."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

MOD = 251
WINDOW = 1 << 20   # the oracle's rows: the last WINDOW of the table


@pytest.fixture(scope="module")
def esc():
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc as m
    return m


@pytest.fixture(scope="module")
def big(esc):
    n = esc.MAX_ROWS
    a = torch.empty(n, dtype=torch.uint8, device="cuda")
    step = 1 << 28
    for s in range(0, n, step):
        e = min(n, s + step)
        a[s:e] = (torch.arange(s, e, dtype=torch.int64, device="cuda") % MOD).to(torch.uint8)
    t = esc.Table([("a", "u8", a)], n)
    host_tail = {"a": a[n - WINDOW:].cpu().numpy()}
    yield n, t, host_tail
    t.close()
    del a
    torch.cuda.empty_cache()


def n_eq(n, v):
    return (n - 1 - v) // MOD + 1 if 0 <= v < min(n, MOD) else 0


CASES = [("a = 7", [7]), ("a = 250", [250]), ("a BETWEEN 3 AND 100", range(3, 101)),
         ("a IN (1, 5, 250)", [1, 5, 250]), ("a > 17 AND a < 120", range(18, 120)),
         ("NOT (a BETWEEN 1 AND 249)", [0, 250]), ("a = 0 OR a >= 200", [0] + list(range(200, 251)))]


def test_counts_at_the_row_limit(esc, big):
    n, t, _ = big
    assert n == (1 << 32) - (1 << 16)
    for text, vals in CASES:
        p = esc.Predicate(t, text)
        assert esc.count(t, p) == sum(n_eq(n, v) for v in vals), text


def test_ordered_ids_at_the_row_limit(esc, big):
    """Every id of `a = 250 OR a = 3` (34.2M rows, the last within 251 rows
    of the table's end) and its projected value; the ids in the last window
    equal the oracle's."""
    n, t, tail = big
    text = "a = 250 OR a = 3"
    p = esc.Predicate(t, text, ("a",))
    c = n_eq(n, 250) + n_eq(n, 3)
    rows = p.alloc_rows(c)
    got, st = esc.esc_selectivity(t.handle, p.handle, rows)
    assert (got, st) == (c, esc.ESC_OK)
    ids = rows[1].to(torch.int64) & 0xFFFFFFFF
    k = torch.arange((c + 1) // 2 + 1, dtype=torch.int64, device="cuda") * MOD
    want = torch.sort(torch.cat([k + 3, k + 250]))[0]
    want = want[want < n]
    assert int(want.numel()) == c
    assert torch.equal(ids, want)
    assert int(ids[-1]) > n - MOD
    assert torch.equal(rows[2][0].to(torch.int64), want % MOD)     # the projected a of each row
    # the oracle on the last window, ids shifted to the table's
    o_ids, _ = oracle.select(text, tail)
    tail_ids = ids[ids >= n - WINDOW].cpu().numpy()
    assert np.array_equal(tail_ids, o_ids.astype(np.int64) + (n - WINDOW))


def test_bitmap_at_the_row_limit(esc, big):
    n, t, tail = big
    text = "a BETWEEN 3 AND 100"
    p = esc.Predicate(t, text)
    words = (n + 31) // 32
    bm = torch.zeros(words, dtype=torch.int32, device="cuda")
    cnt = esc.esc_bitmap_build(t.handle, p.handle, bm)
    assert cnt == sum(n_eq(n, v) for v in range(3, 101))
    last = bm[(n - WINDOW) // 32:].cpu().numpy().view(np.uint32)
    bits = np.unpackbits(last.view(np.uint8), bitorder="little")
    assert np.array_equal(bits, oracle.mark(text, tail).astype(np.uint8))
    del bm


def test_shared_batch_and_noalloc_at_the_row_limit(esc, big):
    n, t, _ = big
    preds = [esc.Predicate(t, text) for text, _ in CASES]
    want = [sum(n_eq(n, v) for v in vals) for _, vals in CASES]
    dev = torch.zeros(len(preds), dtype=torch.int64, device="cuda")
    esc.esc_selectivity_shared_async(t.handle, [p.handle for p in preds], dev)
    assert dev.tolist() == want
    counts, st = esc.esc_selectivity_batch([t.handle] * len(preds), [p.handle for p in preds])
    assert st == esc.ESC_OK and list(counts) == want
    assert esc.esc_selectivity_noalloc(t.handle, preds[0].handle)[0] == want[0]
    # materialising needs nrows/8 bytes of scratch, more than the built-in array
    sel = esc.Predicate(t, "a = 7", ("a",))
    with pytest.raises(esc.EscError) as ei:
        esc.esc_selectivity_noalloc(t.handle, sel.handle, sel.alloc_rows(n_eq(n, 7)))
    assert ei.value.status == esc.ESC_EINVAL


def test_semijoin_at_the_row_limit(esc):
    """Semi-join counts over a fact table of 2^32 - 2^16 rows: fk0 = row mod
    1000 and fk1 = row mod 1024 into two dimensions of 1000 rows (keys
    1000..1023 of fk1 match nothing).  The keys repeat every 128,000 rows, so
    the expected counts are the oracle's nested loop over one period times
    the number of whole periods, plus the oracle over the remaining rows."""
    n = esc.MAX_ROWS
    period = 128_000
    fk = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(2)]
    step = 1 << 28
    for s in range(0, n, step):
        e = min(n, s + step)
        r = torch.arange(s, e, dtype=torch.int64, device="cuda")
        fk[0][s:e] = (r % 1000).to(torch.int32)
        fk[1][s:e] = (r % 1024).to(torch.int32)
        del r
    fact = esc.Table([("fk0", "i32", fk[0]), ("fk1", "i32", fk[1])], n)
    keys = np.arange(1000)
    marks = [(keys % 3 == 0).astype(np.uint8), (keys % 5 != 2).astype(np.uint8)]
    bms = [torch.from_numpy(np.packbits(m, bitorder="little").view(np.uint8).copy()) for m in marks]
    bms = [torch.nn.functional.pad(b, (0, (-b.numel()) % 4)).view(torch.int32).cuda() for b in bms]
    got = esc.esc_semijoin_counts(fact.handle, ["fk0", "fk1"], bms, [1000, 1000])
    r = np.arange(period, dtype=np.int64)
    one = [(r % 1000).astype(np.int32), (r % 1024).astype(np.int32)]
    q, rem = divmod(n, period)
    per = oracle.semijoin_counts(one, marks, [0, 1, 2, 3])
    part = oracle.semijoin_counts([c[:rem] for c in one], marks, [0, 1, 2, 3])
    want = [q * per[s] + part[s] for s in range(4)]
    assert want[0] == n
    assert list(got) == want, (got, want)
    fact.close()
    del fk
    torch.cuda.empty_cache()
