"""The allocation-free entry point gives the same answers as esc_selectivity
and as the oracle.

esc_selectivity_noalloc exists for callers that must not allocate device
memory (an allocator of their own owns the GPU's memory, or cudaMalloc /
cudaFree would synchronise a latency-critical path).  Its scratch is an
array built into the library and shared by every call, so this test calls it
twice in a row on each case: the second call must not see the first call's
leftovers.  The file is named so that pytest collects it last.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def esc():
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc as m
    return m


def _rows_equal(a, b, k):
    return all(torch.equal(x[:k], y[:k]) for x, y in zip([a[1]] + list(a[2]), [b[1]] + list(b[2])))


def test_noalloc_matches_selectivity_twice(esc):
    t = datagen.skewed_table(3_000_017, seed=11, device="cuda")
    tbl = esc.Table.from_datagen(t)
    proj = datagen.SKEWED_PROJECTION
    texts = [p.text for p in datagen.skewed_predicates(200)[::40]] + ["price > 1000000", "FALSE"]
    for text in texts:
        p = esc.Predicate(tbl, text, proj)
        ref_count = esc.count(tbl, p)
        ref = p.alloc_rows(ref_count + 5)
        n_ref, st_ref = esc.esc_selectivity(tbl.handle, p.handle, ref)
        assert n_ref == ref_count and st_ref == esc.ESC_OK
        for _ in range(2):
            n0, st0 = esc.esc_selectivity_noalloc(tbl.handle, p.handle)        # count only
            assert n0 == ref_count and st0 == esc.ESC_OK
            got = p.alloc_rows(ref_count + 5)
            got[1].fill_(-1)
            for c in got[2]:
                c.fill_(-1)
            n1, st1 = esc.esc_selectivity_noalloc(tbl.handle, p.handle, got)
            assert n1 == ref_count and st1 == esc.ESC_OK, text
            assert _rows_equal(got, ref, ref_count), text
    torch.cuda.synchronize()


def test_noalloc_limits(esc):
    # counting needs no per-row scratch: any size works
    t = datagen.single_table(130_000_000, seed=1, device="cuda")
    tbl = esc.Table.from_datagen(t)
    p = esc.Predicate(tbl, "category = 3 AND day < 100", ("key",))
    assert esc.esc_selectivity_noalloc(tbl.handle, p.handle)[0] == esc.count(tbl, p)
    # materialising a table beyond the built-in scratch is refused, not faulted
    with pytest.raises(esc.EscError) as ei:
        esc.esc_selectivity_noalloc(tbl.handle, p.handle, p.alloc_rows(16))
    assert ei.value.status == esc.ESC_EINVAL
    assert "12 MiB" in str(ei.value)


def test_noalloc_matches_oracle(esc):
    """On a small ragged table the count, the ordered ids and the projected
    values equal the oracle's, on two calls in a row."""
    t = datagen.skewed_table(250_003, seed=12, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    proj = datagen.SKEWED_PROJECTION
    for text in [p.text for p in datagen.skewed_predicates(200)[5::50]] + ["udf(price, qty, 97) > 90 OR code7 = 3"]:
        p = esc.Predicate(tbl, text, proj)
        ids, pv = oracle.select(text, host, proj)
        for _ in range(2):
            got = p.alloc_rows(len(ids) + 1)
            n, st = esc.esc_selectivity_noalloc(tbl.handle, p.handle, got)
            assert st == esc.ESC_OK and n == len(ids), text
            assert np.array_equal(got[1][:n].cpu().numpy().view(np.uint32), ids), text
            for name, c in zip(proj, got[2]):
                assert np.array_equal(c[:n].cpu().numpy(), pv[name]), (text, name)


_FRESH = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_1901_01488_gb300 import esc
t = torch.arange(1000, dtype=torch.int32, device="cuda")
tbl = esc.Table([("a", "i32", t)], 1000)
for text, want in (("TRUE", 1000), ("a < 0 AND a > 5", 0)):
    p = esc.Predicate(tbl, text, ("a",))
    n, st = esc.esc_selectivity_noalloc(tbl.handle, p.handle)
    assert (n, st) == (want, esc.ESC_OK), (text, n, st)
    rows = p.alloc_rows(1001)
    n, st = esc.esc_selectivity_noalloc(tbl.handle, p.handle, rows)
    assert (n, st) == (want, esc.ESC_OK), (text, n, st)
    assert torch.equal(rows[1][:n], t[:n]) and torch.equal(rows[2][0][:n], t[:n])
print("ok")
"""


def test_noalloc_constant_predicate_first_in_fresh_process(esc):
    """A constant predicate (folded to TRUE or FALSE by the compiler) as the
    very first call of a process: answered by the constant kernel, launched
    directly, with the right count and rows."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
