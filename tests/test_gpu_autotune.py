"""The autotuner picks a launch shape per class and results never change with it."""
import json

import pytest
import torch

from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_tuning_never_changes_results():
    """Every block shape and tile/unit size gives the oracle's count, ordered
    ids and projected values (single calls, count and materialising)."""
    import numpy as np
    import oracle
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc
    from paper_1901_01488_gb300.autotune import SHAPES, SHAPES_UDF
    t = datagen.skewed_table(3_000_011, seed=60, device="cuda")
    host = t.host()
    tbl = esc.Table.from_datagen(t)
    proj = datagen.SKEWED_PROJECTION
    tiles = ((2048, 16, 64), (4096, 128, 1), (32768, 4096, 8), (256, 16, 3), (32768, 512, 8))
    texts = [pt.text for pt in datagen.skewed_predicates(200)[::25]]
    texts.append("udf(price, qty, 97) > 40 AND code7 IN (1, 2, 5)")
    for text in texts:
        p = esc.Predicate(tbl, text, proj)
        ids, pv = oracle.select(text, host, proj)
        shapes = SHAPES_UDF if "udf" in text else SHAPES
        for k, shape in enumerate(shapes):
            cand = tiles[k % len(tiles)] + shape
            esc.esc_predicate_set_tuning(p.handle, cand)
            assert esc.esc_predicate_get_tuning(p.handle) == cand
            assert esc.count(tbl, p) == len(ids), (text, cand)
            n, got_ids, got_proj = esc.select(tbl, p)
            assert n == len(ids), (text, cand)
            assert np.array_equal(got_ids.cpu().numpy().view(np.uint32), ids), (text, cand)
            for name, c in zip(proj, got_proj):
                assert np.array_equal(c.cpu().numpy(), pv[name]), (text, cand, name)
        if "udf" in text:
            with pytest.raises(esc.EscError):
                esc.esc_predicate_set_tuning(p.handle, (32768, 512, 8, 23, 8))
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
    assert chosen and all(len(v) == 5 for v in chosen.values())
    cache = json.load(open(tmp_path / "tune.json"))
    assert set(cache) == set(chosen)
    k = class_key(tbl, preds[0], False)
    if k in cache:
        assert tuner.apply(tbl, preds[0]) == tuple(cache[k])
    again = Autotuner(esc, str(tmp_path / "tune.json"))
    assert again.cache == tuner.cache


def test_autotuned_batch_matches_oracle(tmp_path):
    """A prepared batch whose launch shapes the tuner chose (its choices
    applied per class) gives the oracle's counts, ordered ids and projected
    values for every sub-query, replayed twice from its CUDA graph."""
    import numpy as np
    import oracle
    from paper_1901_01488_gb300 import esc
    from paper_1901_01488_gb300.autotune import Autotuner, DEFAULT
    sizes = (50_000, 700_003, 3_000_000)
    tabs = [datagen.skewed_table(n, seed=62 + i, device="cuda") for i, n in enumerate(sizes)]
    etabs = [esc.Table.from_datagen(t) for t in tabs]
    hosts = [t.host() for t in tabs]
    work = datagen.batch_workload(36, seed=9, sizes=sizes)
    proj = datagen.SKEWED_PROJECTION
    preds = [esc.Predicate(etabs[ti], p.text, proj) for ti, p in work]
    tuner = Autotuner(esc, str(tmp_path / "tune.json"), repeats=1)
    for k, et in enumerate(etabs):
        mine = [p for (ti, _), p in zip(work, preds) if ti == k]
        tuner.tune(et, mine[0::2], materialise=True)
        tuner.tune(et, mine[1::2], materialise=False)
    applied = []
    expect, rows = [], []
    for j, ((ti, p), pr) in enumerate(zip(work, preds)):
        mat = j % 2 == 0
        applied.append(tuner.apply(etabs[ti], pr, materialise=mat))
        ids, pv = oracle.select(p.text, hosts[ti], proj)
        expect.append((ids, pv))
        rows.append(pr.alloc_rows(len(ids) + 2) if mat else None)
    assert any(a != DEFAULT for a in applied)           # the tuner's choices are really in use
    b = esc.esc_batch_prepare([etabs[ti].handle for ti, _ in work], [p.handle for p in preds], rows)
    dev_counts = torch.zeros(len(work), dtype=torch.int64, device="cuda")
    for _ in range(2):
        for r in rows:
            if r is not None:
                r[1].fill_(-1)
        dev_counts.zero_()
        esc.esc_batch_run(b, dev_counts)
        torch.cuda.synchronize()
        counts = dev_counts.tolist()
        for j, (ids, pv) in enumerate(expect):
            assert counts[j] == len(ids), work[j][1].text
            if rows[j] is not None:
                got = rows[j][1][:len(ids)].cpu().numpy().view(np.uint32)
                assert np.array_equal(got, ids), work[j][1].text
                for name, c in zip(proj, rows[j][2]):
                    assert np.array_equal(c[:len(ids)].cpu().numpy(), pv[name]), (work[j][1].text, name)
    esc.esc_batch_destroy(b)
