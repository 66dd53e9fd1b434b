"""The seeded generator: counter-based, chunk-independent, platform-neutral bits."""
import numpy as np
import torch

from paper_1901_01488_gb300 import datagen


def _splitmix_u64(key: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 (Steele, Lea, Flood 2014) on numpy uint64, written independently."""
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(datagen.GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def test_raw_matches_uint64_reference():
    key = datagen.stream_key(7, 3)
    idx = np.arange(1000, 5000, dtype=np.int64)
    got = datagen.raw_u64(7, 3, 1000, 4000, "cpu").numpy().view(np.uint64)
    assert np.array_equal(got, _splitmix_u64(key, idx))


def test_known_splitmix_vector():
    # Published SplitMix64 output for state seeded at 0: first value 0xE220A8397B1DCDAF.
    z = datagen._mix_py(datagen.GAMMA)
    assert z == 0xE220A8397B1DCDAF


def test_chunk_independent_and_ranges():
    t1 = datagen.single_table(10_000, seed=1)
    t2 = datagen.single_table(20_000, seed=1)
    for c1, c2 in zip(t1.columns, t2.columns):
        assert torch.equal(c1.data, c2.data[:10_000])
    h = t2.host()
    assert h["key"].min() >= 0 and h["key"].max() < (1 << 20)
    assert h["day"].min() >= 0 and h["day"].max() <= 2556
    assert h["price"].min() >= 100 and h["price"].max() <= 10_000_000
    assert h["category"].max() <= 24 and h["category"].dtype == np.uint8


def test_skewed_table_shape_and_correlation():
    t = datagen.skewed_table(200_000, seed=2)
    h = t.host()
    assert t.row_bytes == 32
    assert h["code150"].dtype == np.uint16 and h["code150"].max() <= 149
    eq = np.mean(h["code25"] == (h["code150"] % 25))
    assert 0.7 < eq < 0.76          # 70 % forced + 30 % x 1/25 by chance
    # Zipf(1.1): the most popular key carries a large share of rows
    top = np.bincount(h["key"]).max() / len(h["key"])
    assert top > 0.05


def test_predicates_parse_and_are_seeded():
    import oracle
    ps = datagen.skewed_predicates(50)
    ps2 = datagen.skewed_predicates(50)
    assert [p.text for p in ps] == [p.text for p in ps2]
    for p in ps:
        oracle.parse(p.text)
        assert 1 <= len(p.terms) <= 6


def test_zipf_sampling_matches_the_law():
    """Keys drawn by inverse CDF follow P(rank r) = r^-s / H(n, s): the top
    ranks one by one, and rank buckets [2^k, 2^(k+1)), within 5 sigma of the
    binomial count; the key map is a bijection (exhaustive on a small n)."""
    import math
    n, s, count, salt = 1 << 24, 1.1, 2_000_000, 777
    keys = datagen.zipf_keys(7, 0, 0, count, s, n, "cpu", salt=salt).numpy().astype(np.int64)
    inv = pow(datagen.ZIPF_MULT, -1, n)
    rank = ((keys - salt % n) % n * inv) % n + 1              # 1-based ranks
    h = sum(r ** -s for r in range(1, 2_000_001)) + ((n + 0.5) ** (1 - s) - (2_000_000.5) ** (1 - s)) / (1 - s)
    for r in range(1, 9):                                    # the head, rank by rank
        p = r ** -s / h
        got = np.count_nonzero(rank == r)
        assert abs(got - count * p) < 5 * math.sqrt(count * p * (1 - p)), (r, got, count * p)
    for k in range(0, 24, 3):                                # buckets of ranks
        lo, hi = 1 << k, 1 << (k + 1)
        p = sum(r ** -s for r in range(lo, min(hi, 200_000))) / h if hi <= 200_000 else \
            ((hi - 0.5) ** (1 - s) - (lo - 0.5) ** (1 - s)) / (1 - s) / h
        got = np.count_nonzero((rank >= lo) & (rank < hi))
        assert abs(got - count * p) < 5 * math.sqrt(count * p * (1 - p)) + 1e-4 * count, (k, got, count * p)
    small = 1000 if math.gcd(datagen.ZIPF_MULT, 1000) == 1 else 1001
    ks = datagen.zipf_key_of_rank(torch.arange(small), small, salt).numpy()
    assert sorted(ks.tolist()) == list(range(small))


def test_headline_predicates_test_each_column_once():
    """No two terms of a headline predicate read the same column (two draws
    on one column would mostly be disjoint: a contradiction that reads no
    column at all once compiled), and the generator's aim stays within two
    decades of every target."""
    import math
    for p in datagen.skewed_predicates(200):
        cols = [c for t in p.terms for c in datagen._term_columns(t)]
        assert len(cols) == len(set(cols)), p.text
        assert abs(math.log10(p.est / p.target)) < 2.0, p.text
