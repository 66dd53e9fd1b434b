"""ctypes front end of the C oracle (``esc_oracle.c``) -- TEST INFRASTRUCTURE.

Builds ``liboracle.so`` with the host C compiler when it is missing or older
than its source, flattens the parsed predicate into the C tree-walker's node
array, and calls it on host numpy columns.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .parse import parse

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_K = {"and": 0, "or": 1, "not": 2, "const": 3, "cmp": 4, "between": 5, "in": 6}
_OP = {"=": 0, "!=": 1, "<": 2, "<=": 3, ">": 4, ">=": 5}
_T = {np.dtype(np.int32): 0, np.dtype(np.int64): 1, np.dtype(np.uint8): 2, np.dtype(np.uint16): 3}

ONODE = np.dtype([("kind", np.int32), ("nchild", np.int32), ("op", np.int32), ("neg", np.int32),
                  ("udf", np.int32), ("col", np.int32), ("col2", np.int32), ("pad", np.int32),
                  ("a", np.int64), ("b", np.int64), ("m", np.int64), ("voff", np.int64)])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, plain C99); returns the library path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC],
                           check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_count.argtypes = [P, P, P, P, i64, i64]
        lib.oracle_count.restype = i64
        lib.oracle_select.argtypes = [P, P, P, P, i64, P, i64]
        lib.oracle_select.restype = i64
        lib.oracle_mark.argtypes = [P, P, P, P, i64, P]
        lib.oracle_mark.restype = None
        lib.oracle_semijoin_count.argtypes = [P, ctypes.c_int32, P, P, ctypes.c_uint32, i64, i64]
        lib.oracle_semijoin_count.restype = i64
        _lib = lib
    return _lib


class _Bound:
    """A predicate flattened against one table's column order."""

    def __init__(self, text: str, columns: Dict[str, np.ndarray]):
        ast = parse(text)
        self.names = list(columns)
        self.arrays = [np.ascontiguousarray(columns[n]) for n in self.names]
        for a in self.arrays:
            if a.dtype not in _T:
                raise TypeError(f"oracle: unsupported column dtype {a.dtype}")
        nrows = {len(a) for a in self.arrays}
        if len(nrows) > 1:
            raise ValueError("oracle: columns of different lengths")
        self.nrows = nrows.pop() if nrows else 0
        self.dtypes = np.array([_T[a.dtype] for a in self.arrays], dtype=np.int32)
        self.ptrs = (ctypes.c_void_p * max(1, len(self.arrays)))(
            *[a.ctypes.data for a in self.arrays])
        nodes: List[tuple] = []
        vals: List[int] = []
        self._flatten(ast, nodes, vals)
        self.nodes = np.zeros(len(nodes), dtype=ONODE)
        for i, n in enumerate(nodes):
            self.nodes[i] = n
        self.vals = np.array(vals + [0], dtype=np.int64)

    def _col(self, name: str) -> int:
        try:
            return self.names.index(name)
        except ValueError:
            raise KeyError(f"oracle: unknown column {name!r}") from None

    def _opd(self, o) -> Tuple[int, int, int, int]:
        if o[0] == "col":
            return 0, self._col(o[1]), 0, 1
        return 1, self._col(o[1]), self._col(o[2]), o[3]

    def _flatten(self, e, nodes, vals):
        k = e[0]
        z = dict(kind=_K[k], nchild=0, op=0, neg=0, udf=0, col=0, col2=0, pad=0, a=0, b=0, m=1, voff=0)
        if k in ("and", "or"):
            z["nchild"] = len(e[1])
            nodes.append(tuple(z.values()))
            for c in e[1]:
                self._flatten(c, nodes, vals)
            return
        if k == "not":
            z["nchild"] = 1
            nodes.append(tuple(z.values()))
            self._flatten(e[1], nodes, vals)
            return
        if k == "const":
            z["a"] = int(bool(e[1]))
        elif k == "cmp":
            z["op"] = _OP[e[1]]
            z["udf"], z["col"], z["col2"], z["m"] = self._opd(e[2])
            z["a"] = e[3]
        elif k == "between":
            z["udf"], z["col"], z["col2"], z["m"] = self._opd(e[1])
            z["a"], z["b"], z["neg"] = e[2], e[3], int(e[4])
        elif k == "in":
            z["udf"], z["col"], z["col2"], z["m"] = self._opd(e[1])
            z["nchild"], z["voff"], z["neg"] = len(e[2]), len(vals), int(e[3])
            vals.extend(e[2])
        nodes.append(tuple(z.values()))

    def args(self):
        return (self.nodes.ctypes.data, self.vals.ctypes.data,
                ctypes.cast(self.ptrs, ctypes.c_void_p), self.dtypes.ctypes.data)


def count(text: str, columns: Dict[str, np.ndarray], row0: int = 0,
          row1: Optional[int] = None) -> int:
    """Exact COUNT(*) of rows [row0, row1) satisfying the predicate."""
    b = _Bound(text, columns)
    r1 = b.nrows if row1 is None else row1
    return int(_load().oracle_count(*b.args(), row0, r1))


def count_parallel(text: str, columns: Dict[str, np.ndarray], threads: int,
                   row0: int = 0, row1: Optional[int] = None) -> int:
    """The same count, rows split into `threads` contiguous chunks run concurrently."""
    b = _Bound(text, columns)
    r1 = b.nrows if row1 is None else row1
    lib = _load()
    edges = np.linspace(row0, r1, threads + 1).astype(np.int64)
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda k: lib.oracle_count(*b.args(), int(edges[k]), int(edges[k + 1])),
                            range(threads)))
    return int(sum(parts))


def select(text: str, columns: Dict[str, np.ndarray],
           proj: Sequence[str] = ()) -> Tuple[np.ndarray, Dict[str, np.ndarray]]:
    """(ascending qualifying row ids as uint32, {name: projected values})."""
    b = _Bound(text, columns)
    lib = _load()
    n = lib.oracle_select(*b.args(), b.nrows, None, 0)
    ids = np.empty(max(1, n), dtype=np.uint32)
    n2 = lib.oracle_select(*b.args(), b.nrows, ids.ctypes.data, n)
    assert n2 == n
    ids = ids[:n]
    return ids, {p: np.ascontiguousarray(columns[p][ids]) for p in proj}


def mark(text: str, columns: Dict[str, np.ndarray]) -> np.ndarray:
    """uint8 flag per row (= per dense key): 1 where the predicate holds."""
    b = _Bound(text, columns)
    out = np.zeros(max(1, b.nrows), dtype=np.uint8)
    _load().oracle_mark(*b.args(), b.nrows, out.ctypes.data)
    return out[:b.nrows]


def semijoin_counts(fk: Sequence[np.ndarray], marks: Sequence[np.ndarray],
                    subsets: Sequence[int], row0: int = 0, row1: Optional[int] = None,
                    threads: int = 1) -> Dict[int, int]:
    """{subset mask: exact semijoin count} by a nested loop over rows and dimensions."""
    fk = [np.ascontiguousarray(f, dtype=np.int32) for f in fk]
    marks = [np.ascontiguousarray(m, dtype=np.uint8) for m in marks]
    nd = len(fk)
    n = len(fk[0]) if nd else 0
    r1 = n if row1 is None else row1
    fkp = (ctypes.c_void_p * nd)(*[f.ctypes.data for f in fk])
    mp = (ctypes.c_void_p * nd)(*[m.ctypes.data for m in marks])
    rows = np.array([len(m) for m in marks], dtype=np.int64)
    lib = _load()
    edges = np.linspace(row0, r1, threads + 1).astype(np.int64)
    out = {}
    for s in subsets:
        def part(k, s=s):
            return lib.oracle_semijoin_count(ctypes.cast(fkp, ctypes.c_void_p), nd,
                                             ctypes.cast(mp, ctypes.c_void_p),
                                             rows.ctypes.data, s, int(edges[k]), int(edges[k + 1]))
        if threads == 1:
            out[s] = int(part(0))
        else:
            with ThreadPoolExecutor(threads) as ex:
                out[s] = int(sum(ex.map(part, range(threads))))
    return out
