"""CPU oracle for exact selectivity computation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never calls it, and it never calls the product: the two share
only the seeded input generator, which holds none of the method's arithmetic.

What it computes -- the plain definitions of the paper's selectivity
sub-query (Shin, Rusu, Suhan, "Exact Selectivity Computation for Modern
In-Memory Database Query Optimization", Sec. 1 and Sec. 2):

* ``count(text, table)``   -- SELECT COUNT(*) FROM R WHERE <predicate>, row at
  a time, by a C tree walker over the parsed predicate (``esc_oracle.c``).
* ``select(text, table, proj)`` -- the qualifying row ids in ascending order and
  their projected columns: the sub-query result that ESC materialises as a
  temporary table (Sec. 1, Sec. 2.1), with the projection pushed down (Sec. 2).
* ``mark(text, dim)`` -- qualifying flag per dense dimension key.
* ``semijoin_counts(fk, marks, dim_rows, subsets)`` -- the exact fact-table
  cardinality after joining with each subset of filtered dimensions (the
  COUNT(*) foreign-key join queries of Sec. 3.1), as a nested loop.
* ``pyeval`` -- the same definition in pure Python for exhaustive checks on
  tiny tables.
* ``mlp`` -- an FP64 forward/backward of the selectivity surrogate network.

Pins (tests/test_oracle_pins.py): exhaustive brute force on tiny tables
against SQLite (an independent SQL engine) and the pure-Python evaluator; a
hand-worked 10-row table; closed forms from numpy (bincount bins, sorted
searches); invariants (|A or B| = |A| + |B| - |A and B|, NOT P = N - P,
monotone ranges, AND never raises a count, semijoin of the empty set = N,
single-dimension semijoin = sum over keys of mark x frequency).
"""
from __future__ import annotations

from .parse import parse, columns_of, OracleParseError  # noqa: F401
from .native import count, select, mark, semijoin_counts, count_parallel  # noqa: F401
