"""The batched workload at its full size, as the benchmark runs it: 512
sub-queries over six tables of 10K to 60M rows, every one materialising
(key, day, price), prepared in 10 waves and replayed from its CUDA graph.

The oracle decides every count (threaded over row chunks). It decides every
ordered row list and projected value on the tables of up to 2M rows. On the
larger tables, the rows are checked by properties that hold at any size
(strictly increasing ids in range, projected values equal to the table's
values at those ids) and by 64 sampled rows per sub-query that the oracle
decides one by one against membership in the returned ids.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_full_size_batch_in_waves_matches_oracle():
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc
    sizes = datagen.BATCH_TABLE_ROWS
    tabs = [datagen.skewed_table(n, seed=30 + i, device="cuda") for i, n in enumerate(sizes)]
    etabs = [esc.Table.from_datagen(t) for t in tabs]
    work = datagen.batch_workload(512, seed=3, sizes=sizes)
    proj = datagen.SKEWED_PROJECTION
    preds = [esc.Predicate(etabs[ti], p.text, proj) for ti, p in work]
    hosts = [t.host() for t in tabs]
    threads = max(2, os.cpu_count() or 2)
    want = [oracle.count_parallel(p.text, hosts[ti], threads) for ti, p in work]
    rows = [p.alloc_rows(c + 1) for p, c in zip(preds, want)]
    b = esc.esc_batch_prepare_waves([etabs[ti].handle for ti, _ in work], [p.handle for p in preds], rows,
                                    waves=10)
    dc = torch.zeros(len(work), dtype=torch.int64, device="cuda")
    rng = np.random.default_rng(12)
    for rep in range(2):
        for r in rows:
            r[1].fill_(-1)
        dc.zero_()
        esc.esc_batch_run(b, dc)
        torch.cuda.synchronize()
        assert dc.tolist() == want
        if rep == 0:
            continue                      # the second replay is checked in full
        for j, ((ti, pd), n) in enumerate(zip(work, want)):
            ids = rows[j][1][:n]
            if sizes[ti] <= 2_000_000:
                exp_ids, pv = oracle.select(pd.text, hosts[ti], proj)
                assert np.array_equal(ids.cpu().numpy().view(np.uint32), exp_ids), pd.text
                for name, c in zip(proj, rows[j][2]):
                    assert np.array_equal(c[:n].cpu().numpy(), pv[name]), (pd.text, name)
                continue
            ids64 = ids.to(torch.int64) & 0xffffffff
            if n:
                assert int(ids64[0]) >= 0 and int(ids64[-1]) < sizes[ti], pd.text
                assert bool((ids64[1:] > ids64[:-1]).all()), pd.text
                for name, c in zip(proj, rows[j][2]):
                    assert torch.equal(c[:n], tabs[ti].col(name).data.index_select(0, ids64)), (pd.text, name)
            sample = np.sort(rng.choice(sizes[ti], 64, replace=False))
            sub = {name: col[sample] for name, col in hosts[ti].items()}
            member = np.zeros(64, dtype=bool)
            member[oracle.select(pd.text, sub)[0].astype(np.int64)] = True
            got = torch.isin(torch.from_numpy(sample).cuda(), ids64).cpu().numpy()
            assert np.array_equal(got, member), pd.text
    esc.esc_batch_destroy(b)
