"""Star-schema semi-join counts at the full 600M-row size, checked against
the oracle's nested loop (all host cores) on several dimension subsets."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1901_01488_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_star_full_size_subsets():
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc
    fact = datagen.star_fact(600_000_000, seed=4, device="cuda")
    ftab = esc.Table.from_datagen(fact)
    texts = datagen.star_dim_predicates(4)
    bms, marks = [], []
    for d, n in enumerate(datagen.STAR_DIM_ROWS):
        dim = datagen.star_dim(d, n, seed=4, device="cuda")
        dtab = esc.Table.from_datagen(dim)
        p = esc.Predicate(dtab, texts[d])
        bm = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")
        esc.esc_bitmap_build(dtab.handle, p.handle, bm)
        bms.append(bm)
        marks.append(oracle.mark(texts[d], dim.host()))
    got = esc.esc_semijoin_counts(ftab.handle, [f"fk{d}" for d in range(4)], bms, list(datagen.STAR_DIM_ROWS))
    assert got[0] == 600_000_000
    fk = [fact.col(f"fk{d}").numpy() for d in range(4)]
    threads = max(1, os.cpu_count() or 1)
    exp = oracle.semijoin_counts(fk, marks, [1, 2, 4, 8, 5, 15], threads=threads)
    for s, v in exp.items():
        assert got[s] == v, (s, got[s], v)
    # every subset count is monotone under inclusion
    for s in range(16):
        for t in range(16):
            if s & t == s:
                assert got[t] <= got[s]
