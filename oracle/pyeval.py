"""Pure-Python, row-at-a-time evaluation of a predicate AST (tiny inputs only).

Test infrastructure (see ``oracle/__init__.py``).  The definition it follows
is the paper's selectivity sub-query (Sec. 2): the exact number of rows of R
for which the selection predicate holds, and the rows themselves with the
projected attributes (Sec. 1, Sec. 2.1: the sub-query result is materialised
as a temporary table).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

_I64 = 1 << 64


def _wrap64(x: int) -> int:
    x %= _I64
    return x - _I64 if x >= (1 << 63) else x


def _c_rem(p: int, m: int) -> int:
    """C99 remainder: the sign follows the dividend, quotient truncated to zero."""
    r = abs(p) % m
    return -r if p < 0 else r


def operand_value(opd, row: Dict[str, int]) -> int:
    if opd[0] == "col":
        return row[opd[1]]
    _, a, b, m = opd
    return _c_rem(_wrap64(row[a] * row[b]), m)


def holds(e, row: Dict[str, int]) -> bool:
    k = e[0]
    if k == "and":
        return all([holds(c, row) for c in e[1]])
    if k == "or":
        return any([holds(c, row) for c in e[1]])
    if k == "not":
        return not holds(e[1], row)
    if k == "const":
        return bool(e[1])
    if k == "cmp":
        _, op, opd, c = e
        x = operand_value(opd, row)
        return {"=": x == c, "!=": x != c, "<": x < c, "<=": x <= c,
                ">": x > c, ">=": x >= c}[op]
    if k == "between":
        _, opd, lo, hi, neg = e
        x = operand_value(opd, row)
        return (lo <= x <= hi) != neg
    if k == "in":
        _, opd, vals, neg = e
        x = operand_value(opd, row)
        return (x in vals) != neg
    raise ValueError(k)


def select(ast, columns: Dict[str, Sequence[int]], nrows: int) -> List[int]:
    """Row ids (ascending) of the rows for which the predicate holds."""
    names = list(columns)
    out = []
    for i in range(nrows):
        row = {n: int(columns[n][i]) for n in names}
        if holds(ast, row):
            out.append(i)
    return out


def count(ast, columns, nrows: int) -> int:
    return len(select(ast, columns, nrows))
