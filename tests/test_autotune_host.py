"""Host logic of the autotuner (autotune.py) and the tuning entry points of
the C ABI, no GPU: range checks, class keys, the choice per class, the JSON
cache and its use.  Timing is replaced by a deterministic cost."""
import json

import numpy as np
import pytest

from _helpers import as_columns
from paper_1901_01488_gb300 import autotune
from paper_1901_01488_gb300 import build as esc_build


@pytest.fixture(scope="module")
def esc():
    esc_build.build()
    from paper_1901_01488_gb300 import esc as m
    return m


def _table(esc, n):
    rng = np.random.default_rng(2)
    cols = {"k": rng.integers(0, 1000, n).astype(np.int32), "p": rng.integers(0, 10**6, n).astype(np.int64),
            "c": rng.integers(0, 25, n).astype(np.uint8)}
    return esc.Table(as_columns(cols), n)


def test_tuning_ranges_and_defaults(esc):
    t = _table(esc, 1000)
    p = esc.Predicate(t, "k < 5")
    assert esc.esc_predicate_get_tuning(p.handle) == autotune.DEFAULT
    for good in ((256, 16, 1), (32768, 4096, 64), (8192, 128, 16)):
        esc.esc_predicate_set_tuning(p.handle, good)
        assert esc.esc_predicate_get_tuning(p.handle) == good
    for bad in ((0, 512, 8), (300, 512, 8), (32768 + 256, 512, 8), (128, 512, 8),
                (8192, 15, 8), (8192, 4097, 8), (8192, 512, 0), (8192, 512, 65)):
        with pytest.raises(esc.EscError):
            esc.esc_predicate_set_tuning(p.handle, bad)
        assert esc.esc_predicate_get_tuning(p.handle) == (8192, 128, 16)    # unchanged
    esc.esc_predicate_set_tuning(p.handle, None)
    assert esc.esc_predicate_get_tuning(p.handle) == autotune.DEFAULT
    for cand in autotune.CANDIDATES:                                        # every candidate is valid
        esc.esc_predicate_set_tuning(p.handle, cand)


def test_class_key(esc):
    t = _table(esc, 3000)                                   # log2(3000) = 11.55 -> r11
    assert autotune.class_key(t, esc.Predicate(t, "k < 5"), False) == "r11_b4_c"
    assert autotune.class_key(t, esc.Predicate(t, "k < 5 AND p > 3 AND c = 1"), True) == "r11_b13_m"
    assert autotune.class_key(t, esc.Predicate(t, "k < 5 OR k > 900"), False) == "r11_b4_c"   # one read
    assert autotune.read_bytes_per_row(esc.Predicate(t, "TRUE")) == 0


class _FakeEsc:
    """Records the tuning calls the tuner makes (the real library is not
    needed for the choice logic)."""

    def __init__(self):
        self.calls = []

    def esc_predicate_set_tuning(self, handle, cand):
        self.calls.append((handle, cand))


class _CostTuner(autotune.Autotuner):
    """Timing replaced by a cost: per class, the candidate named in `best`
    is fastest; every call is recorded."""

    def __init__(self, fake, best, **kw):
        super().__init__(fake, **kw)
        self.best = best
        self.timed = []

    def _time(self, table, preds, rows, cand):
        key = autotune.class_key(table, preds[0], False)
        self.timed.append((key, cand))
        return 1.0 if cand == self.best[key] else 2.0 + autotune.CANDIDATES.index(cand)


def test_choice_cache_and_apply(esc, tmp_path):
    t = _table(esc, 5000)
    preds = [esc.Predicate(t, x) for x in ("k < 5", "k > 7", "k < 5 AND p > 3", "c IN (1, 2)", "k = 1 AND p = 2")]
    keys = sorted({autotune.class_key(t, p, False) for p in preds})
    assert keys == ["r12_b12_c", "r12_b1_c", "r12_b4_c"]
    best = {"r12_b4_c": autotune.CANDIDATES[3], "r12_b12_c": autotune.CANDIDATES[6], "r12_b1_c": autotune.CANDIDATES[0]}
    cache = tmp_path / "tune.json"
    fake = _FakeEsc()
    tuner = _CostTuner(fake, best, cache_path=str(cache))
    chosen = tuner.tune(t, preds)
    assert chosen == best
    assert {k for k, _ in tuner.timed} == set(keys) and len(tuner.timed) == len(keys) * len(autotune.CANDIDATES)
    # the samples' tuning is restored to the defaults afterwards
    assert all(cand is None for _, cand in fake.calls[-len(preds):])
    assert {k: tuple(v) for k, v in json.loads(cache.read_text()).items()} == best
    # a second tuner reads the cache: nothing is timed again, apply() uses the choices
    fake2 = _FakeEsc()
    again = _CostTuner(fake2, best, cache_path=str(cache))
    assert again.tune(t, preds) == {} and again.timed == []
    for p in preds:
        assert again.apply(t, p) == best[autotune.class_key(t, p, False)]
    assert [c for _, c in fake2.calls] == [best[autotune.class_key(t, p, False)] for p in preds]
    # an untuned class (materialising) gets the defaults
    assert again.apply(t, preds[0], materialise=True) == autotune.DEFAULT
