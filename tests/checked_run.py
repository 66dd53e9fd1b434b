"""Runs the sub-query paths with canary words after every output buffer and
checks each result against the oracle (a test helper, run as a subprocess by
tests/test_gpu_checked.py, with ESC_CHECKED=1 to load the checked build).

Exits non-zero (with a message) on the first failure: a wrong count, id or
projected value, a canary word overwritten, or a status other than the
expected one (the checked build reports ESC_EBOUNDS for any out-of-range
index its kernels meet).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np
import torch

import oracle
from paper_1901_01488_gb300 import datagen, esc

CANARY = 64          # elements after each output buffer
PATTERN = 0x5A       # byte pattern of the canary elements

want_checked = os.environ.get("ESC_CHECKED") == "1"
assert esc.esc_build_checked() == want_checked, "the wrong library was loaded"


def buffers(pred, capacity):
    ids = torch.full((capacity + CANARY,), 0, dtype=torch.int32, device="cuda")
    cols = [torch.zeros(capacity + CANARY, dtype=esc.TORCH_DTYPE[pred.table.dtype(p)], device="cuda")
            for p in pred.proj]
    for t in [ids] + cols:
        t.view(torch.uint8)[capacity * t.element_size():].fill_(PATTERN)
    return ids, cols


def canaries_intact(capacity, ids, cols):
    for t in [ids] + cols:
        tail = t.view(torch.uint8)[capacity * t.element_size():]
        if not bool((tail == PATTERN).all()):
            return False
    return True


def check_select(tbl, host, text, proj, capacity=None, tuning=None):
    p = esc.Predicate(tbl, text, proj)
    if tuning is not None:
        esc.esc_predicate_set_tuning(p.handle, tuning)
    exp_ids, exp_proj = oracle.select(text, host, proj)
    n = len(exp_ids)
    cap = n if capacity is None else capacity
    ids, cols = buffers(p, cap)
    got, st = esc.esc_selectivity(tbl.handle, p.handle, (cap, ids, cols))
    assert got == n, (text, got, n)
    assert st == (esc.ESC_OK if cap >= n else esc.ESC_ETRUNC), (text, st)
    k = min(n, cap)
    assert np.array_equal(ids[:k].cpu().numpy().view(np.uint32), exp_ids[:k]), text
    for name, c in zip(proj, cols):
        g = c[:k].cpu().numpy()
        if host[name].dtype == np.uint16:
            g = g.view(np.uint16)
        assert np.array_equal(g, exp_proj[name][:k]), (text, name)
    assert canaries_intact(cap, ids, cols), ("canary overwritten", text, cap)
    assert esc.count(tbl, p) == n, text


def main():
    texts = ["day < 1500", "category IN (1, 2, 3) OR price > 5000000", "TRUE", "FALSE",
             datagen.SINGLE_TABLE_PREDICATE, "udf(price, day, 97) > 40", "category = 3",
             "NOT (key BETWEEN 1000 AND 900000) AND category != 4"]
    proj = ("key", "day", "price", "category")
    for n in (0, 1, 17, 255, 256, 257, 4097, 65537, 100_003, 300_001):
        t = datagen.single_table(n, seed=5, device="cuda")
        host = t.host()
        tbl = esc.Table.from_datagen(t)
        for text in texts:
            check_select(tbl, host, text, proj)
            if n > 0:
                n_sel = len(oracle.select(text, host)[0])
                for cap in sorted({0, 1, n_sel // 2, max(0, n_sel - 1)}):
                    if cap < n_sel:
                        check_select(tbl, host, text, proj, capacity=cap)   # truncated
    # the skewed table: every column type, the headline predicates
    t = datagen.skewed_table(1_000_003, seed=7, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    for pd in datagen.skewed_predicates(200)[::10]:
        check_select(tbl, host, pd.text, datagen.SKEWED_PROJECTION)
        check_select(tbl, host, pd.text, datagen.SKEWED_PROJECTION, capacity=7)
    # every block shape of the scan kernel, small tiles and units too
    from paper_1901_01488_gb300.autotune import SHAPES, SHAPES_UDF
    texts = [pd.text for pd in datagen.skewed_predicates(200)[5::25]]
    texts.append("udf(price, qty, 97) > 40 AND code7 IN (1, 2, 5)")
    for j, text in enumerate(texts):
        for k, shape in enumerate(SHAPES_UDF if "udf" in text else SHAPES):
            tile = ((2048, 16, 64), (32768, 512, 8), (256, 16, 3))[(j + k) % 3]
            check_select(tbl, host, text, datagen.SKEWED_PROJECTION, tuning=tile + shape)
    # a batch mixing materialising and count-only sub-queries
    ps = [esc.Predicate(tbl, pd.text, datagen.SKEWED_PROJECTION) for pd in datagen.skewed_predicates(40, seed0=900)]
    exp = [oracle.select(p.text, host, datagen.SKEWED_PROJECTION) for p in ps]
    rows = []
    for j, (p, (ids_e, _)) in enumerate(zip(ps, exp)):
        rows.append((len(ids_e),) + buffers(p, len(ids_e)) if j % 2 == 0 else None)
    counts, st = esc.esc_selectivity_batch([tbl.handle] * len(ps), [p.handle for p in ps], rows)
    assert st == esc.ESC_OK, st
    for j, (p, (ids_e, pv)) in enumerate(zip(ps, exp)):
        assert counts[j] == len(ids_e), p.text
        if rows[j] is not None:
            cap, ids, cols = rows[j]
            assert np.array_equal(ids[:cap].cpu().numpy().view(np.uint32), ids_e), p.text
            assert canaries_intact(cap, ids, cols), ("canary overwritten in a batch", p.text)
    # bitmaps and semi-join counts, edge keys included
    dim = datagen.single_table(70_001, seed=8, device="cuda")
    dh = dim.host()
    dtbl = esc.Table.from_datagen(dim)
    dp = esc.Predicate(dtbl, "category < 9 AND day > 300")
    words = (70_001 + 31) // 32
    bm = torch.zeros(words + CANARY, dtype=torch.int32, device="cuda")
    bm.view(torch.uint8)[words * 4:].fill_(PATTERN)
    cnt = esc.esc_bitmap_build(dtbl.handle, dp.handle, bm)
    mark = oracle.mark(dp.text, dh)
    assert cnt == int(mark.sum())
    assert bool((bm.view(torch.uint8)[words * 4:] == PATTERN).all()), "canary after the bitmap"
    rng = np.random.default_rng(3)
    fk = rng.integers(-3, 70_004, 500_003).astype(np.int32)
    fk[:4] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, -1, 70_001]
    fact = esc.Table([("fk", "i32", torch.from_numpy(fk).cuda())], len(fk))
    got = esc.esc_semijoin_counts(fact.handle, ["fk"], [bm[:words]], [70_001])
    want = oracle.semijoin_counts([fk], [mark], [0, 1])
    assert got[1] == want[1] and got[0] == want[0] == len(fk), (got, want)
    # a dimension too large for shared memory (probed in place) beside a small one
    big = 1_000_003
    bw = rng.integers(0, 2**32, (big + 31) // 32, dtype=np.uint64).astype(np.uint32)
    bmark = np.unpackbits(bw.view(np.uint8), bitorder="little")[:big].astype(np.uint8)
    fk2 = rng.integers(-3, big + 4, 500_003).astype(np.int32)
    fk2[:4] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, -1, big]
    fact2 = esc.Table([("fk", "i32", torch.from_numpy(fk2).cuda()), ("fk2", "i32", torch.from_numpy(fk).cuda())],
                      len(fk))
    got = esc.esc_semijoin_counts(fact2.handle, ["fk", "fk2"], [torch.from_numpy(bw.view(np.int32).copy()).cuda(),
                                                               bm[:words]], [big, 70_001])
    want = oracle.semijoin_counts([fk2, fk], [bmark, mark], [0, 1, 2, 3])
    assert got == [want[s] for s in range(4)], (got, want)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
