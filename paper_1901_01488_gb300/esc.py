"""Python binding of libesc (ctypes): argument marshalling only.

Every function here has the name of the C entry point it calls
(include/esc.h) and does nothing but convert arguments; all the work of the
selectivity sub-query runs in the library's CUDA kernels.  If the library has
not been built, importing this module raises: there is no fallback.

PyTorch supplies device memory and streams: columns and output buffers are
torch tensors on the current CUDA device, passed by data pointer.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# ESC_CHECKED=1 loads the checked build (kernels that test every index they
# use and report ESC_EBOUNDS); the release build otherwise
LIB_PATH = os.path.join(_HERE, "libesc_checked.so" if os.environ.get("ESC_CHECKED") == "1" else "libesc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); "
                      "run `python -m paper_1901_01488_gb300.build`")
_lib = ctypes.CDLL(LIB_PATH)

ESC_OK, ESC_EINVAL, ESC_ETYPE, ESC_ENOMEM, ESC_ETRUNC, ESC_ETIMEOUT, ESC_EBUSY, ESC_ECUDA, ESC_EBOUNDS = range(9)
DTYPE_CODE = {"i32": 0, "i64": 1, "u8": 2, "u16": 3}
WIDTH = {"i32": 4, "i64": 8, "u8": 1, "u16": 2}
MAX_ROWS = (1 << 32) - (1 << 16)   # ESC_MAX_ROWS: rows a table may hold
TORCH_DTYPE = {"i32": torch.int32, "i64": torch.int64, "u8": torch.uint8, "u16": torch.int16}


class esc_column(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("dtype", ctypes.c_int32), ("data", ctypes.c_void_p)]


class esc_tuning(ctypes.Structure):
    _fields_ = [("max_tile_rows", ctypes.c_uint32), ("max_unit_kb", ctypes.c_uint32),
                ("units_per_sm", ctypes.c_int32), ("consumer_warps", ctypes.c_uint16),
                ("rows_per_pass", ctypes.c_uint16)]


class esc_rows(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_uint64), ("row_ids", ctypes.c_void_p),
                ("proj", ctypes.POINTER(ctypes.c_void_p)), ("written", ctypes.c_uint64)]


_P = ctypes.c_void_p
_S = ctypes.c_int
_sig = {
    "esc_table_create": ([ctypes.POINTER(esc_column), ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(_P)], _S),
    "esc_table_destroy": ([_P], _S),
    "esc_table_nrows": ([_P], ctypes.c_uint64),
    "esc_predicate_compile": ([_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_char_p), ctypes.c_int32,
                               ctypes.POINTER(_P)], _S),
    "esc_predicate_destroy": ([_P], _S),
    "esc_predicate_compile_many": ([_P, ctypes.POINTER(ctypes.c_char_p), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_char_p), ctypes.c_int32, ctypes.POINTER(_P),
                                    ctypes.c_int32], _S),
    "esc_predicate_explain": ([_P, ctypes.c_char_p, ctypes.c_uint64], _S),
    "esc_predicate_set_tuning": ([_P, ctypes.POINTER(esc_tuning)], _S),
    "esc_predicate_get_tuning": ([_P, ctypes.POINTER(esc_tuning)], _S),
    "esc_selectivity": ([_P, _P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(esc_rows), _P], _S),
    "esc_selectivity_async": ([_P, _P, _P, ctypes.POINTER(esc_rows), _P], _S),
    "esc_selectivity_noalloc": ([_P, _P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(esc_rows), _P], _S),
    "esc_batch_prepare": ([ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(esc_rows),
                           ctypes.POINTER(_P)], _S),
    "esc_batch_prepare_waves": ([ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(esc_rows),
                                 ctypes.c_int32, ctypes.POINTER(_P)], _S),
    "esc_batch_run": ([_P, _P, _P, _P], _S),
    "esc_batch_destroy": ([_P], _S),
    "esc_selectivity_batch": ([ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(esc_rows), _P], _S),
    "esc_bitmap_build": ([_P, _P, _P, ctypes.POINTER(ctypes.c_uint64), _P], _S),
    "esc_semijoin_counts": ([_P, ctypes.POINTER(ctypes.c_char_p), ctypes.c_int32, ctypes.POINTER(_P),
                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _P], _S),
    "esc_last_error": ([], ctypes.c_char_p),
    "esc_status_string": ([_S], ctypes.c_char_p),
    "esc_udf_magic": ([ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32),
                       ctypes.POINTER(ctypes.c_int32)], _S),
    "esc_selftest_wait_timeout": ([ctypes.c_uint64, _P], _S),
    "esc_timestamp": ([_P, _P], _S),
    "esc_selectivity_shared_async": ([_P, ctypes.POINTER(_P), ctypes.c_int32, _P, _P], _S),
    "esc_selectivity_batch_async": ([ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int32,
                                     ctypes.POINTER(esc_rows), _P, _P, _P], _S),
    "esc_debug_fail_allocs": ([ctypes.c_int32], _S),
    "esc_debug_write_units": ([ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32)], _S),
    "esc_build_checked": ([ctypes.POINTER(ctypes.c_int32)], _S),
    "esc_mlp_forward": ([_P, ctypes.c_uint64, _P, _P, _P, _P], _S),
    "esc_mlp_grad": ([_P, _P, ctypes.c_uint64, _P, _P, _P, _P, _P], _S),
    "esc_mlp_adam": ([_P, _P, _P, _P, _P, ctypes.c_uint64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, ctypes.c_int32, _P], _S),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_sig)


class EscError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.esc_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_lib.esc_status_string(status).decode()}: {msg}")


def _check(status: int, where: str, ok=(ESC_OK,)) -> int:
    if status not in ok:
        raise EscError(status, where)
    return status


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ------------------------------------------------------------------ thin wrappers
def esc_table_create(columns: Sequence[Tuple[str, str, torch.Tensor]], nrows: int) -> int:
    arr = (esc_column * len(columns))()
    for i, (name, dtype, t) in enumerate(columns):
        arr[i].name = name.encode()
        arr[i].dtype = DTYPE_CODE.get(dtype, 99)
        arr[i].data = t.data_ptr() if t.numel() else None
    out = _P()
    _check(_lib.esc_table_create(arr, len(columns), nrows, ctypes.byref(out)), "esc_table_create")
    return out.value


def esc_table_destroy(handle: int) -> None:
    _lib.esc_table_destroy(handle)


def esc_table_nrows(handle: int) -> int:
    return int(_lib.esc_table_nrows(handle))


def esc_predicate_compile(table: int, text: str, proj: Sequence[str] = ()) -> int:
    names = (ctypes.c_char_p * max(1, len(proj)))(*[p.encode() for p in proj])
    out = _P()
    _check(_lib.esc_predicate_compile(table, text.encode(), names, len(proj), ctypes.byref(out)),
           "esc_predicate_compile")
    return out.value


def esc_predicate_destroy(pred: int) -> None:
    _lib.esc_predicate_destroy(pred)


def esc_predicate_compile_many(table: int, texts: Sequence[str], proj: Sequence[str] = (),
                               threads: int = 0) -> List[int]:
    """Handles of the compiled texts (the caller destroys each)."""
    n = len(texts)
    arr = (ctypes.c_char_p * max(1, n))(*[t.encode() for t in texts])
    names = (ctypes.c_char_p * max(1, len(proj)))(*[p.encode() for p in proj])
    out = (_P * max(1, n))()
    _check(_lib.esc_predicate_compile_many(table, arr, n, names, len(proj), out, threads),
           "esc_predicate_compile_many")
    return [out[i] for i in range(n)]


def esc_predicate_explain(pred: int) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_lib.esc_predicate_explain(pred, buf, len(buf)), "esc_predicate_explain")
    return buf.value.decode()


def esc_predicate_set_tuning(pred: int, tuning: Optional[Tuple[int, ...]]) -> None:
    """tuning = (max_tile_rows, max_unit_kb, units_per_sm[, consumer_warps,
    rows_per_pass]) -- the block shape (0, 0), automatic, when left out -- or
    None for the defaults."""
    if tuning is None:
        _check(_lib.esc_predicate_set_tuning(pred, None), "esc_predicate_set_tuning")
        return
    if len(tuning) not in (3, 5):
        raise ValueError("tuning is (max_tile_rows, max_unit_kb, units_per_sm[, consumer_warps, rows_per_pass])")
    shape = tuple(tuning[3:5]) if len(tuning) == 5 else (0, 0)
    t = esc_tuning(tuning[0], tuning[1], tuning[2], shape[0], shape[1])
    _check(_lib.esc_predicate_set_tuning(pred, ctypes.byref(t)), "esc_predicate_set_tuning")


def esc_predicate_get_tuning(pred: int) -> Tuple[int, int, int, int, int]:
    """(max_tile_rows, max_unit_kb, units_per_sm, consumer_warps, rows_per_pass)."""
    t = esc_tuning()
    _check(_lib.esc_predicate_get_tuning(pred, ctypes.byref(t)), "esc_predicate_get_tuning")
    return t.max_tile_rows, t.max_unit_kb, t.units_per_sm, t.consumer_warps, t.rows_per_pass


def _rows_struct(capacity: int, row_ids: Optional[torch.Tensor], proj: Sequence[torch.Tensor]):
    ptrs = (ctypes.c_void_p * max(1, len(proj)))(*[p.data_ptr() for p in proj])
    r = esc_rows(capacity, row_ids.data_ptr() if row_ids is not None else None,
                 ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), 0)
    return r, ptrs


def esc_selectivity(table: int, pred: int, rows=None, stream=None) -> Tuple[int, int]:
    """Returns (count, status); status is ESC_OK or ESC_ETRUNC.  rows is None or
    (capacity, row_ids tensor, [projected tensors])."""
    cnt = ctypes.c_uint64()
    if rows is None:
        st = _lib.esc_selectivity(table, pred, ctypes.byref(cnt), None, _stream(stream))
        _check(st, "esc_selectivity")
        return cnt.value, st
    r, keep = _rows_struct(*rows)
    st = _lib.esc_selectivity(table, pred, ctypes.byref(cnt), ctypes.byref(r), _stream(stream))
    _check(st, "esc_selectivity", ok=(ESC_OK, ESC_ETRUNC))
    return cnt.value, st


def esc_selectivity_noalloc(table: int, pred: int, rows=None, stream=None) -> Tuple[int, int]:
    """Allocation-free esc_selectivity (scratch built into the library).
    Returns (count, status); status is ESC_OK or ESC_ETRUNC."""
    cnt = ctypes.c_uint64()
    if rows is None:
        st = _lib.esc_selectivity_noalloc(table, pred, ctypes.byref(cnt), None, _stream(stream))
        _check(st, "esc_selectivity_noalloc")
        return cnt.value, st
    r, keep = _rows_struct(*rows)
    st = _lib.esc_selectivity_noalloc(table, pred, ctypes.byref(cnt), ctypes.byref(r), _stream(stream))
    _check(st, "esc_selectivity_noalloc", ok=(ESC_OK, ESC_ETRUNC))
    return cnt.value, st


def esc_selectivity_async(table: int, pred: int, dev_count: torch.Tensor, rows=None, stream=None) -> None:
    if rows is None:
        _check(_lib.esc_selectivity_async(table, pred, dev_count.data_ptr(), None, _stream(stream)),
               "esc_selectivity_async")
        return
    r, keep = _rows_struct(*rows)
    _check(_lib.esc_selectivity_async(table, pred, dev_count.data_ptr(), ctypes.byref(r), _stream(stream)),
           "esc_selectivity_async")


def _rows_array(rows):
    """list of None | (capacity, ids, proj) -> (esc_rows array, keep-alive list)."""
    arr = (esc_rows * len(rows))()
    keep = []
    for i, r in enumerate(rows):
        if r is None:
            arr[i] = esc_rows(0, None, None, 0)
        else:
            s, k = _rows_struct(*r)
            arr[i] = s
            keep.append(k)
    return arr, keep


def esc_batch_prepare(tables: Sequence[int], preds: Sequence[int], rows=None) -> int:
    n = len(tables)
    ta = (_P * n)(*tables)
    pa = (_P * n)(*preds)
    out = _P()
    if rows is None:
        _check(_lib.esc_batch_prepare(ta, pa, n, None, ctypes.byref(out)), "esc_batch_prepare")
    else:
        arr, keep = _rows_array(rows)
        _check(_lib.esc_batch_prepare(ta, pa, n, arr, ctypes.byref(out)), "esc_batch_prepare")
    return out.value


def esc_batch_prepare_waves(tables: Sequence[int], preds: Sequence[int], rows=None, waves: int = 1) -> int:
    n = len(tables)
    ta = (_P * n)(*tables)
    pa = (_P * n)(*preds)
    out = _P()
    if rows is None:
        _check(_lib.esc_batch_prepare_waves(ta, pa, n, None, waves, ctypes.byref(out)), "esc_batch_prepare_waves")
    else:
        arr, keep = _rows_array(rows)
        _check(_lib.esc_batch_prepare_waves(ta, pa, n, arr, waves, ctypes.byref(out)), "esc_batch_prepare_waves")
    return out.value


def esc_batch_run(batch: int, dev_counts: Optional[torch.Tensor], dev_done_ns: Optional[torch.Tensor] = None,
                  stream=None) -> None:
    _check(_lib.esc_batch_run(batch, dev_counts.data_ptr() if dev_counts is not None else None,
                              dev_done_ns.data_ptr() if dev_done_ns is not None else None, _stream(stream)),
           "esc_batch_run")


def esc_batch_destroy(batch: int) -> None:
    _lib.esc_batch_destroy(batch)


def esc_selectivity_batch(tables: Sequence[int], preds: Sequence[int], rows=None, stream=None) -> Tuple[List[int], int]:
    n = len(tables)
    ta = (_P * n)(*tables)
    pa = (_P * n)(*preds)
    counts = (ctypes.c_uint64 * n)()
    if rows is None:
        st = _lib.esc_selectivity_batch(ta, pa, n, counts, None, _stream(stream))
    else:
        arr, keep = _rows_array(rows)
        st = _lib.esc_selectivity_batch(ta, pa, n, counts, arr, _stream(stream))
    _check(st, "esc_selectivity_batch", ok=(ESC_OK, ESC_ETRUNC))
    return list(counts), st


def esc_selectivity_batch_async(tables: Sequence[int], preds: Sequence[int], dev_counts: torch.Tensor,
                                rows=None, dev_done_ns: Optional[torch.Tensor] = None, stream=None) -> None:
    n = len(tables)
    ta = (_P * n)(*tables)
    pa = (_P * n)(*preds)
    done = dev_done_ns.data_ptr() if dev_done_ns is not None else None
    if rows is None:
        _check(_lib.esc_selectivity_batch_async(ta, pa, n, None, dev_counts.data_ptr(), done, _stream(stream)),
               "esc_selectivity_batch_async")
    else:
        arr, keep = _rows_array(rows)
        _check(_lib.esc_selectivity_batch_async(ta, pa, n, arr, dev_counts.data_ptr(), done, _stream(stream)),
               "esc_selectivity_batch_async")


def esc_selectivity_shared_async(table: int, preds: Sequence[int], dev_counts: torch.Tensor, stream=None) -> None:
    """Counts of many predicates of one table in one pass over it (shared scan)."""
    n = len(preds)
    pa = (_P * n)(*preds)
    _check(_lib.esc_selectivity_shared_async(table, pa, n, dev_counts.data_ptr(), _stream(stream)),
           "esc_selectivity_shared_async")


def esc_bitmap_build(dim: int, pred: int, dev_bitmap: torch.Tensor, stream=None) -> int:
    cnt = ctypes.c_uint64()
    _check(_lib.esc_bitmap_build(dim, pred, dev_bitmap.data_ptr() if dev_bitmap.numel() else None,
                                 ctypes.byref(cnt), _stream(stream)), "esc_bitmap_build")
    return cnt.value


def esc_semijoin_counts(fact: int, fk_cols: Sequence[str], bitmaps: Sequence[torch.Tensor],
                        dim_rows: Sequence[int], stream=None) -> List[int]:
    nd = len(fk_cols)
    names = (ctypes.c_char_p * nd)(*[c.encode() for c in fk_cols])
    bms = (_P * nd)(*[b.data_ptr() if b is not None else None for b in bitmaps])
    rows = (ctypes.c_uint64 * nd)(*dim_rows)
    out = (ctypes.c_uint64 * (1 << nd))()
    _check(_lib.esc_semijoin_counts(fact, names, nd, bms, rows, out, _stream(stream)), "esc_semijoin_counts")
    return list(out)


def esc_udf_magic(d: int) -> Tuple[int, int, int]:
    m = ctypes.c_uint64()
    s1 = ctypes.c_int32()
    s2 = ctypes.c_int32()
    _check(_lib.esc_udf_magic(d, ctypes.byref(m), ctypes.byref(s1), ctypes.byref(s2)), "esc_udf_magic")
    return m.value, s1.value, s2.value


def esc_selftest_wait_timeout(limit_ns: int, stream=None) -> int:
    return _lib.esc_selftest_wait_timeout(limit_ns, _stream(stream))


def esc_timestamp(dev_ns: torch.Tensor, stream=None) -> None:
    _check(_lib.esc_timestamp(dev_ns.data_ptr(), _stream(stream)), "esc_timestamp")


MLP_PARAMS = 24961


def esc_mlp_forward(x_bf16: torch.Tensor, w_bf16: torch.Tensor, params: torch.Tensor, y: torch.Tensor,
                    stream=None) -> None:
    _check(_lib.esc_mlp_forward(x_bf16.data_ptr(), x_bf16.shape[0], w_bf16.data_ptr(), params.data_ptr(),
                                y.data_ptr(), _stream(stream)), "esc_mlp_forward")


def esc_mlp_grad(x_bf16: torch.Tensor, target: torch.Tensor, w_bf16: torch.Tensor, params: torch.Tensor,
                 grad: torch.Tensor, loss_sum: torch.Tensor, stream=None) -> None:
    _check(_lib.esc_mlp_grad(x_bf16.data_ptr(), target.data_ptr(), x_bf16.shape[0], w_bf16.data_ptr(),
                             params.data_ptr(), grad.data_ptr(), loss_sum.data_ptr(), _stream(stream)),
           "esc_mlp_grad")


def esc_mlp_adam(params: torch.Tensor, w_bf16: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
                 lr: float, step: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 stream=None) -> None:
    _check(_lib.esc_mlp_adam(params.data_ptr(), w_bf16.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(),
                             params.numel(), lr, beta1, beta2, eps, step, _stream(stream)), "esc_mlp_adam")


def esc_debug_fail_allocs(n: int) -> None:
    _check(_lib.esc_debug_fail_allocs(n), "esc_debug_fail_allocs")


def esc_debug_write_units(nrows: int, slots: int) -> Tuple[int, int, int]:
    """(groups per compaction unit, units, group-to-unit reciprocal) of a
    materialising call on `nrows` rows with `slots` write-kernel blocks
    resident (0: a batch's full-size units)."""
    out = (ctypes.c_uint32 * 3)()
    _check(_lib.esc_debug_write_units(nrows, slots, out), "esc_debug_write_units")
    return out[0], out[1], out[2]


def esc_build_checked() -> bool:
    flag = ctypes.c_int32(0)
    _check(_lib.esc_build_checked(ctypes.byref(flag)), "esc_build_checked")
    return bool(flag.value)


def esc_last_error() -> str:
    return _lib.esc_last_error().decode(errors="replace")


# ------------------------------------------------------------------ convenience
class Table:
    """Owns an esc_table handle over device columns (keeps the tensors alive)."""

    def __init__(self, columns: Sequence[Tuple[str, str, torch.Tensor]], nrows: int):
        self.columns = [(n, d, t) for n, d, t in columns]
        self.nrows = nrows
        self.handle = esc_table_create(self.columns, nrows)

    @classmethod
    def from_datagen(cls, table) -> "Table":
        return cls([(c.name, c.dtype, c.data) for c in table.columns], table.nrows)

    def dtype(self, name: str) -> str:
        for n, d, _ in self.columns:
            if n == name:
                return d
        raise KeyError(name)

    def close(self):
        if self.handle:
            esc_table_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Predicate:
    """A predicate compiled against a Table, with its projection."""

    def __init__(self, table: Table, text: str, proj: Sequence[str] = ()):
        self.table = table
        self.text = text
        self.proj = tuple(proj)
        self.handle = esc_predicate_compile(table.handle, text, self.proj)

    def explain(self) -> str:
        return esc_predicate_explain(self.handle)

    def alloc_rows(self, capacity: int, device="cuda"):
        ids = torch.empty(max(1, capacity), dtype=torch.int32, device=device)
        cols = [torch.empty(max(1, capacity), dtype=TORCH_DTYPE[self.table.dtype(p)], device=device)
                for p in self.proj]
        return capacity, ids, cols

    def close(self):
        if self.handle:
            esc_predicate_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PredicateSet:
    """Many predicates compiled against one Table in one call (host threads),
    with one projection; `handles` in the order of the texts."""

    def __init__(self, table: Table, texts: Sequence[str], proj: Sequence[str] = (), threads: int = 0):
        self.table = table
        self.proj = tuple(proj)
        self.handles = esc_predicate_compile_many(table.handle, list(texts), self.proj, threads)

    def __len__(self) -> int:
        return len(self.handles)

    def close(self):
        for h in self.handles:
            esc_predicate_destroy(h)
        self.handles = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count(table: Table, pred: Predicate, stream=None) -> int:
    """Exact COUNT(*) of the selectivity sub-query."""
    return esc_selectivity(table.handle, pred.handle, None, stream)[0]


def select(table: Table, pred: Predicate, capacity: Optional[int] = None, stream=None):
    """(count, row ids, [projected columns]) of the materialised sub-query.

    With capacity None the count is taken first and the buffers sized to it.
    """
    if capacity is None:
        capacity = count(table, pred, stream)
    rows = pred.alloc_rows(capacity)
    n, st = esc_selectivity(table.handle, pred.handle, rows, stream)
    k = min(n, capacity)
    return n, rows[1][:k], [c[:k] for c in rows[2]]
