"""Host logic of the serving loop (serve.py), no GPU: admission by device
memory, wave grouping into shared passes and a batch, the memory estimate,
arrivals and the latency summary."""
from collections import deque

import numpy as np
import pytest

from paper_1901_01488_gb300.serve import (Request, admit, latency_summary, no_gc_pauses, poisson_arrivals,
                                          request_bytes, wave_groups)


def _reqs(spec):
    """spec: list of (table, materialise?) -> requests in arrival order."""
    return [Request(i, t, f"x < {i}", arrival=i * 1e-4, proj=("a",) if m else (), capacity=10 if m else 0)
            for i, (t, m) in enumerate(spec)]


def test_admission_in_order_within_budget_and_batch_size():
    sizes = [300, 200, 600, 100, 100]
    pend = deque(_reqs([(0, True)] * 5))
    size = lambda r: sizes[r.rid]
    batch, nbytes = admit(pend, in_flight=0, budget=1000, max_batch=10, size=size)
    assert [r.rid for r in batch] == [0, 1] and nbytes == 500     # + 600 > 1000: stops at request 2
    assert [r.rid for r in pend] == [2, 3, 4]                       # the rest waits, in order
    batch, nbytes = admit(pend, in_flight=500, budget=1000, max_batch=10, size=size)
    assert batch == [] and nbytes == 0                              # 500 + 600 > 1000: head of line waits
    batch, _ = admit(pend, in_flight=0, budget=1000, max_batch=2, size=size)
    assert [r.rid for r in batch] == [2, 3]                         # max_batch
    # a request larger than the whole budget runs alone, once nothing is in flight
    big = deque(_reqs([(0, True)] * 2))
    batch, nbytes = admit(big, in_flight=1, budget=10, max_batch=10, size=lambda r: 50)
    assert batch == []
    batch, nbytes = admit(big, in_flight=0, budget=10, max_batch=10, size=lambda r: 50)
    assert [r.rid for r in batch] == [0] and nbytes == 50 and len(big) == 1


def test_admission_work_cap():
    pend = deque(_reqs([(0, False)] * 6))
    rows = [100, 300, 50, 700, 10, 10]
    w = lambda r: rows[r.rid]
    size = lambda r: 1
    batch, _ = admit(pend, 0, 1000, 10, size, w, 400)
    assert [r.rid for r in batch] == [0, 1]                         # 100 + 300; + 50 > 400
    batch, _ = admit(pend, 0, 1000, 10, size, w, 400)
    assert [r.rid for r in batch] == [2]                            # 50 + 700 > 400
    batch, _ = admit(pend, 0, 1000, 10, size, w, 400)
    assert [r.rid for r in batch] == [3]                            # above the cap: a wave of its own
    batch, _ = admit(pend, 0, 1000, 10, size, w, 400)
    assert [r.rid for r in batch] == [4, 5] and not pend
    # no cap: only the batch size and the budget
    pend = deque(_reqs([(0, False)] * 6))
    batch, _ = admit(pend, 0, 1000, 10, size, w, None)
    assert len(batch) == 6


def test_admission_never_exceeds_the_budget_when_requests_fit():
    rng = np.random.default_rng(4)
    for _ in range(200):
        n = int(rng.integers(1, 40))
        sizes = rng.integers(1, 200, n).tolist()
        pend = deque(_reqs([(0, True)] * n))
        budget, in_flight = int(rng.integers(200, 2000)), int(rng.integers(0, 200))
        batch, nbytes = admit(pend, in_flight, budget, max_batch=int(rng.integers(1, 50)), size=lambda r: sizes[r.rid])
        assert nbytes == sum(sizes[r.rid] for r in batch)
        assert in_flight + nbytes <= budget
        assert [r.rid for r in batch] + [r.rid for r in pend] == list(range(n))   # order kept, nothing lost


def test_wave_groups():
    # tables interleave: 0 has 3 count requests, 1 has 2, 2 has 3 but one materialises
    spec = [(0, False), (1, False), (0, False), (2, False), (2, True), (1, False), (0, False), (2, False), (2, False)]
    batch = _reqs(spec)
    groups, rest = wave_groups(batch, shared_min=3)
    assert [[r.rid for r in g] for g in groups] == [[0, 2, 6], [3, 7, 8]]   # one pass per table, arrival order
    assert [r.rid for r in rest] == [1, 4, 5]                               # too few, or materialising
    assert sorted(r.rid for g in groups for r in g) + [r.rid for r in rest] == [0, 2, 3, 6, 7, 8, 1, 4, 5]
    groups, rest = wave_groups(batch, shared_min=100)
    assert groups == [] and [r.rid for r in rest] == list(range(len(spec)))
    groups, rest = wave_groups(batch, shared_min=1)
    assert all(not r.proj for g in groups for r in g) and [r.rid for r in rest] == [4]


def test_request_bytes():
    w = {"a": 4, "b": 8}
    count_only = Request(0, 0, "TRUE", 0.0)
    assert request_bytes(60_000_000, count_only, w) == 4096      # a compiled query is ~3.7 KB
    r = Request(0, 0, "TRUE", 0.0, proj=("a", "b"), capacity=1000)
    for n in (1, 255, 256, 65536, 65537, 1_000_000, 8_000_000, 60_000_000, 600_000_000):
        # the bitmap rounded to a whole tile (<= 32768 rows), the unit words
        # (compaction units filling whole waves of 152 SMs x 4 blocks), the outputs
        groups, slots = (n + 255) // 256, 152 * 4
        waves = max(1, -(-groups // (256 * slots)))
        ug = min(256, max(1, -(-groups // (waves * slots))))
        need = (n + 32767) // 8 + 16 * -(-groups // ug) + 1000 * (4 + 12)
        assert request_bytes(n, r, w) >= need
        assert request_bytes(n, r, w) - need <= 16384 + 16 * 1024


def test_poisson_arrivals_and_latency_summary():
    t = poisson_arrivals(200_000, 20_000.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert np.mean(np.diff(t)) == pytest.approx(1 / 20_000.0, rel=0.02)
    reqs = [Request(i, 0, "TRUE", arrival=i * 1e-3) for i in range(100)]
    for i, r in enumerate(reqs):
        r.done = r.arrival + (i + 1) * 1e-4          # latencies 0.1 .. 10 ms
    s = latency_summary(reqs)
    assert s["p50_ms"] == pytest.approx(5.05) and s["max_ms"] == pytest.approx(10.0)
    assert s["p99_ms"] == pytest.approx(np.percentile(np.arange(1, 101) * 0.1, 99))
    assert s["throughput_per_s"] == pytest.approx(100 / (reqs[-1].done - reqs[0].arrival))


def test_no_gc_pauses_restores_the_setting():
    import gc
    assert gc.isenabled()
    with no_gc_pauses():
        assert not gc.isenabled()
    assert gc.isenabled()
    gc.disable()
    try:
        with no_gc_pauses():
            assert not gc.isenabled()
        assert not gc.isenabled()                 # left as it was
    finally:
        gc.enable()
