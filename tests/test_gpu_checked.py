"""Stand-ins for a memory checker (the sanitizer is not available here):

* the checked build (libesc_checked.so, compiled with -DESC_CHECKED) tests
  every index its kernels use -- stage slices, program and constant-pool
  entries, result bytes, bitmap words, compaction units, gathered rows,
  staging slots, semi-join words -- and reports ESC_EBOUNDS instead of
  touching memory out of range.  The sub-query paths (tail sizes, truncated
  outputs, every column type, a batch, bitmaps and semi-joins with edge
  keys) run under it with canary words after every output buffer: results
  equal the oracle's, no check fires, no canary is overwritten;
* the same run with the release build;
* allocation failures injected on the host return ESC_ENOMEM cleanly, and
  the next call works.
No kernel traps, faults or hangs on purpose.
"""
import os
import subprocess
import sys

import pytest
import torch

from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def esc():
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc as m
    return m


def _run(checked: bool):
    env = dict(os.environ)
    env["ESC_CHECKED"] = "1" if checked else "0"
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-3000:] + r.stderr[-3000:]


def test_checked_build_with_canaries(esc):
    _run(checked=True)


def test_release_build_with_canaries(esc):
    _run(checked=False)


def test_injected_allocation_failures(esc):
    t = datagen.single_table(100_000, seed=4, device="cuda")
    tbl = esc.Table.from_datagen(t)
    p = esc.Predicate(tbl, "day < 1000", ("key",))
    n = esc.count(tbl, p)
    # a single call: its scratch allocation fails
    esc.esc_debug_fail_allocs(1)
    with pytest.raises(esc.EscError) as ei:
        esc.count(tbl, p)
    assert ei.value.status == esc.ESC_ENOMEM and "injected" in str(ei.value)
    assert esc.count(tbl, p) == n                        # the injection is used up; the next call works
    # a materialising call, an asynchronous call and a batch
    esc.esc_debug_fail_allocs(3)
    with pytest.raises(esc.EscError) as ei:
        esc.select(tbl, p, capacity=n)
    assert ei.value.status == esc.ESC_ENOMEM
    dc = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(esc.EscError) as ei:
        esc.esc_selectivity_async(tbl.handle, p.handle, dc, None)
    assert ei.value.status == esc.ESC_ENOMEM
    with pytest.raises(esc.EscError) as ei:
        esc.esc_batch_prepare([tbl.handle], [p.handle])
    assert ei.value.status == esc.ESC_ENOMEM
    # semi-join counts
    fact = esc.Table([("fk", "i32", torch.arange(1000, dtype=torch.int32, device="cuda"))], 1000)
    bm = torch.full((32,), -1, dtype=torch.int32, device="cuda")
    esc.esc_debug_fail_allocs(1)
    with pytest.raises(esc.EscError) as ei:
        esc.esc_semijoin_counts(fact.handle, ["fk"], [bm], [1000])
    assert ei.value.status == esc.ESC_ENOMEM
    assert esc.esc_semijoin_counts(fact.handle, ["fk"], [bm], [1000]) == [1000, 1000]
    # everything works again
    esc.esc_debug_fail_allocs(0)
    got = esc.select(tbl, p)
    assert got[0] == n
    counts, st = esc.esc_selectivity_batch([tbl.handle], [p.handle])
    assert counts == [n] and st == esc.ESC_OK
    torch.cuda.synchronize()
