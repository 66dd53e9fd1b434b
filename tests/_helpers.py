"""Seeded random tables and predicates shared by the tests (test helpers)."""
import numpy as np
import torch

def host_table(n=5000, seed=3):
    rng = np.random.default_rng(seed)
    cols = {
        "a": rng.integers(-50, 50, n).astype(np.int32),
        "b": rng.integers(0, 256, n).astype(np.uint8),
        "c": rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64),
        "d": rng.integers(0, 65536, n).astype(np.uint16),
        "e": rng.integers(-(1 << 31), (1 << 31) - 1, n).astype(np.int32),
    }
    cols["c"][:5] = [np.iinfo(np.int64).min, np.iinfo(np.int64).max, -1, 0, 1]
    cols["e"][:3] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, 0]
    return cols



DT = {np.dtype(np.int32): "i32", np.dtype(np.int64): "i64", np.dtype(np.uint8): "u8", np.dtype(np.uint16): "u16"}


def as_columns(cols, device="cpu"):
    """numpy columns -> (name, dtype, tensor) triples for esc.Table."""
    out = []
    for k, v in cols.items():
        a = v.view(np.int16) if v.dtype == np.uint16 else v
        out.append((k, DT[v.dtype], torch.from_numpy(np.ascontiguousarray(a)).to(device)))
    return out


def random_preds(count=400, seed=17):
    rng = np.random.default_rng(seed)
    names = ["a", "b", "c", "d", "e"]
    edge = [0, 1, -1, 255, 256, 65535, 65536, 2**31 - 1, -2**31, 2**31, 2**63 - 1, -2**63, 7, -50, 49]

    def const():
        return int(rng.choice(edge)) if rng.random() < 0.4 else int(rng.integers(-300, 300))

    def opd():
        if rng.random() < 0.2:
            x, y = rng.choice(names, 2)
            return f"udf({x}, {y}, {int(rng.choice([1, 2, 7, 97, 65535, 65536, 1000003, 2**62 + 1]))})"
        return str(rng.choice(names))

    def atom():
        k = rng.integers(5)
        o = opd()
        if k == 0:
            return f"{o} {rng.choice(['=', '!=', '<', '<=', '>', '>=', '<>', '=='])} {const()}"
        if k == 1:
            lo = const()
            hi = max(-2**63, min(2**63 - 1, lo + int(rng.integers(-5, 400))))
            return f"{o} {'NOT ' if rng.random() < 0.3 else ''}BETWEEN {lo} AND {hi}"
        if k == 2:
            vals = ", ".join(str(const()) for _ in range(int(rng.integers(0, 17))))
            return f"{o} {'NOT ' if rng.random() < 0.3 else ''}IN ({vals})"
        if k == 3:
            return str(rng.choice(["TRUE", "FALSE"]))
        return f"{o} >= {const()}"

    def expr(depth):
        if depth == 0 or rng.random() < 0.35:
            return atom()
        k = rng.integers(3)
        if k == 0:
            return "NOT (" + expr(depth - 1) + ")"
        j = " AND " if k == 1 else " OR "
        return "(" + j.join(expr(depth - 1) for _ in range(int(rng.integers(2, 4)))) + ")"

    return [expr(3) for _ in range(count)]


