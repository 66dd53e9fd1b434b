"""The autotuner picks a launch shape per class and results never change with it."""
import json

import pytest
import torch

from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_tuning_never_changes_results(esc_mod=None):
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc
    t = datagen.skewed_table(3_000_011, seed=60, device="cuda")
    tbl = esc.Table.from_datagen(t)
    for pt in datagen.skewed_predicates(200)[::25]:
        p = esc.Predicate(tbl, pt.text, datagen.SKEWED_PROJECTION)
        ref = esc.select(tbl, p)
        for cand in ((2048, 16, 64), (4096, 128, 1), (32768, 4096, 8), (256, 16, 3)):
            esc.esc_predicate_set_tuning(p.handle, cand)
            assert esc.esc_predicate_get_tuning(p.handle) == cand
            got = esc.select(tbl, p)
            assert got[0] == ref[0] and torch.equal(got[1], ref[1])
            for a, b in zip(got[2], ref[2]):
                assert torch.equal(a, b)
        with pytest.raises(esc.EscError):
            esc.esc_predicate_set_tuning(p.handle, (300, 512, 8))


def test_autotuner_caches_choices(tmp_path):
    from paper_1901_01488_gb300 import esc
    from paper_1901_01488_gb300.autotune import Autotuner, class_key
    t = datagen.skewed_table(4_000_000, seed=61, device="cuda")
    tbl = esc.Table.from_datagen(t)
    preds = [esc.Predicate(tbl, p.text) for p in datagen.skewed_predicates(40, seed0=7000)]
    tuner = Autotuner(esc, str(tmp_path / "tune.json"), repeats=2)
    chosen = tuner.tune(tbl, preds[:12])
    assert chosen and all(len(v) == 3 for v in chosen.values())
    cache = json.load(open(tmp_path / "tune.json"))
    assert set(cache) == set(chosen)
    k = class_key(tbl, preds[0], False)
    if k in cache:
        assert tuner.apply(tbl, preds[0]) == tuple(cache[k])
    again = Autotuner(esc, str(tmp_path / "tune.json"))
    assert again.cache == tuner.cache
