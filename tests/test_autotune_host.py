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
    for good in ((256, 16, 1), (32768, 4096, 64), (8192, 128, 16)):     # block shape left out: automatic
        esc.esc_predicate_set_tuning(p.handle, good)
        assert esc.esc_predicate_get_tuning(p.handle) == good + (0, 0)
    for shape in autotune.SHAPES:                                          # every compiled shape, no udf
        esc.esc_predicate_set_tuning(p.handle, (4096, 64, 2) + shape)
        assert esc.esc_predicate_get_tuning(p.handle) == (4096, 64, 2) + shape
    esc.esc_predicate_set_tuning(p.handle, (8192, 128, 16))
    for bad in ((0, 512, 8), (300, 512, 8), (32768 + 256, 512, 8), (128, 512, 8),
                (8192, 15, 8), (8192, 4097, 8), (8192, 512, 0), (8192, 512, 65),
                (8192, 512, 8, 16, 16), (8192, 512, 8, 19, 4), (8192, 512, 8, 0, 16), (8192, 512, 8, 15, 0),
                (8192, 512, 8, 23, 16), (8192, 512, 8, 32, 8)):
        with pytest.raises(esc.EscError):
            esc.esc_predicate_set_tuning(p.handle, bad)
        assert esc.esc_predicate_get_tuning(p.handle) == (8192, 128, 16, 0, 0)    # unchanged
    with pytest.raises(ValueError):
        esc.esc_predicate_set_tuning(p.handle, (8192, 512, 8, 19))            # a shape needs both numbers
    esc.esc_predicate_set_tuning(p.handle, None)
    assert esc.esc_predicate_get_tuning(p.handle) == autotune.DEFAULT
    for tile in autotune.TILE_CANDIDATES:                                  # every candidate is valid
        for shape in autotune.SHAPES:
            esc.esc_predicate_set_tuning(p.handle, tile + shape)
    # a program with a udf runs only the shapes with the udf path
    u = esc.Predicate(t, "udf(k, p, 7) > 3 AND c = 1")
    for shape in autotune.SHAPES:
        if shape in autotune.SHAPES_UDF:
            esc.esc_predicate_set_tuning(u.handle, (32768, 512, 8) + shape)
            assert esc.esc_predicate_get_tuning(u.handle)[3:] == shape
        else:
            with pytest.raises(esc.EscError):
                esc.esc_predicate_set_tuning(u.handle, (32768, 512, 8) + shape)


def test_class_key(esc):
    t = _table(esc, 3000)                                   # log2(3000) = 11.55 -> r11
    assert autotune.class_key(t, esc.Predicate(t, "k < 5"), False) == "r11_b4_c"
    assert autotune.class_key(t, esc.Predicate(t, "k < 5 AND p > 3 AND c = 1"), True) == "r11_b13_m"
    assert autotune.class_key(t, esc.Predicate(t, "k < 5 OR k > 900"), False) == "r11_b4_c"   # one read
    assert autotune.class_key(t, esc.Predicate(t, "udf(k, p, 7) > 3"), False) == "r11_b12_u_c"
    assert autotune.shapes_for("r11_b12_u_c") == autotune.SHAPES_UDF
    assert autotune.shapes_for("r11_b12_c") == autotune.SHAPES
    assert autotune.read_bytes_per_row(esc.Predicate(t, "TRUE")) == 0


class _FakeEsc:
    """Records the tuning calls the tuner makes (the real library is not
    needed for the choice logic)."""

    def __init__(self):
        self.calls = []

    def esc_predicate_set_tuning(self, handle, cand):
        self.calls.append((handle, cand))


class _CostTuner(autotune.Autotuner):
    """Timing replaced by a cost: per class, the block shape and the
    tile/unit sizes of `best` are the fastest (each slower candidate adds its
    rank); every call is recorded."""

    def __init__(self, fake, best, **kw):
        super().__init__(fake, **kw)
        self.best = best
        self.timed = []

    def _time(self, table, preds, rows, cand):
        key = autotune.class_key(table, preds[0], False)
        self.timed.append((key, cand))
        b = self.best[key]
        shapes = autotune.shapes_for(key)
        cost = 0.0 if cand[3:] == b[3:] else 1.0 + shapes.index(cand[3:])
        cost += 0.0 if cand[:3] == b[:3] else 0.5 + autotune.TILE_CANDIDATES.index(cand[:3])
        return 1.0 + cost


def test_choice_cache_and_apply(esc, tmp_path):
    t = _table(esc, 5000)
    preds = [esc.Predicate(t, x) for x in ("k < 5", "k > 7", "k < 5 AND p > 3", "c IN (1, 2)", "k = 1 AND p = 2",
                                           "udf(k, p, 7) > 3")]
    keys = sorted({autotune.class_key(t, p, False) for p in preds})
    assert keys == ["r12_b12_c", "r12_b12_u_c", "r12_b1_c", "r12_b4_c"]
    T, S, SU = autotune.TILE_CANDIDATES, autotune.SHAPES, autotune.SHAPES_UDF
    best = {"r12_b4_c": T[3] + S[3], "r12_b12_c": T[6] + S[2], "r12_b1_c": T[0] + S[0], "r12_b12_u_c": T[5] + SU[1]}
    cache = tmp_path / "tune.json"
    fake = _FakeEsc()
    tuner = _CostTuner(fake, best, cache_path=str(cache))
    chosen = tuner.tune(t, preds)
    assert chosen == best
    # per class: every shape it can run at the default sizes, then every
    # tile/unit candidate at the fastest shape (the default sizes once)
    assert {k for k, _ in tuner.timed} == set(keys)
    for k in keys:
        timed = [c for kk, c in tuner.timed if kk == k]
        assert len(timed) == len(set(timed)) == len(autotune.shapes_for(k)) + len(T) - 1
        assert all(c[3:] in autotune.shapes_for(k) for c in timed)      # a udf class never runs a lean shape
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


def test_cache_without_block_shape(tmp_path):
    """A cache written before block shapes were tuned reads as the automatic shape."""
    cache = tmp_path / "old.json"
    cache.write_text(json.dumps({"r12_b4_c": [8192, 128, 16]}))
    tuner = autotune.Autotuner(_FakeEsc(), cache_path=str(cache))
    assert tuner.cache == {"r12_b4_c": (8192, 128, 16, 0, 0)}
