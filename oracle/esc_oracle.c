/*
 * Plain, slow, row-at-a-time CPU oracle for exact selectivity computation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library.  It shares no code,
 * header or table with the CUDA library; its inputs are host copies of the
 * same seeded columns.
 *
 * What it computes (each is the plain definition, written out):
 *  - oracle_count: the answer of the selectivity sub-query
 *      SELECT COUNT(*) FROM R WHERE <predicate>          (paper Sec. 2)
 *    by walking the predicate tree once per row.
 *  - oracle_select: the ascending ids of the qualifying rows, i.e. the
 *    materialised sub-query result (Sec. 1, Sec. 2.1) before projection.
 *  - oracle_semijoin_count: |{ i : for every d in S, 0 <= fk_d[i] < D_d and
 *    dim_d row fk_d[i] qualifies }|, the exact cardinality of the fact table
 *    joined with the filtered dimensions on dense keys (the COUNT(*) join
 *    queries of Sec. 3.1), as a nested loop over rows and dimensions.
 *
 * Semantics fixed here (the paper is silent on them):
 *  - every column value is widened to int64 (signed types sign-extend,
 *    unsigned types zero-extend) and compared with int64 constants;
 *  - BETWEEN lo AND hi is inclusive at both ends, empty when lo > hi;
 *  - udf(a, b, m) = (a * b) mod m with the product wrapping in two's
 *    complement 64-bit arithmetic and the remainder truncated toward zero
 *    (C99 '%'), m > 0;
 *  - AND/OR/NOT are plain boolean connectives, no NULLs.
 */
#include <stdint.h>
#include <stddef.h>

enum { K_AND = 0, K_OR = 1, K_NOT = 2, K_CONST = 3, K_CMP = 4, K_BETWEEN = 5, K_IN = 6 };
enum { OP_EQ = 0, OP_NE = 1, OP_LT = 2, OP_LE = 3, OP_GT = 4, OP_GE = 5 };
enum { T_I32 = 0, T_I64 = 1, T_U8 = 2, T_U16 = 3 };

/* One node of the predicate tree, children following their parent (prefix order). */
typedef struct {
    int32_t kind;    /* K_* */
    int32_t nchild;  /* AND/OR/NOT: number of children; IN: number of values */
    int32_t op;      /* CMP: OP_* */
    int32_t neg;     /* BETWEEN / IN: 1 for NOT BETWEEN / NOT IN */
    int32_t udf;     /* 0: operand is column `col`; 1: udf(col, col2, m) */
    int32_t col;
    int32_t col2;
    int32_t pad;
    int64_t a;       /* CMP constant, BETWEEN low bound, CONST truth value */
    int64_t b;       /* BETWEEN high bound */
    int64_t m;       /* udf modulus */
    int64_t voff;    /* IN: first value in vals[] */
} onode;

typedef struct {
    const void *const *cols;
    const int32_t *dtypes;
    const int64_t *vals;
} otable;

static int64_t column_value(const otable *t, int32_t c, int64_t i)
{
    switch (t->dtypes[c]) {
    case T_I32: return (int64_t)((const int32_t *)t->cols[c])[i];
    case T_I64: return ((const int64_t *)t->cols[c])[i];
    case T_U8:  return (int64_t)((const uint8_t *)t->cols[c])[i];
    case T_U16: return (int64_t)((const uint16_t *)t->cols[c])[i];
    }
    return 0;
}

static int64_t operand_value(const otable *t, const onode *n, int64_t i)
{
    int64_t x = column_value(t, n->col, i);
    if (!n->udf) return x;
    int64_t y = column_value(t, n->col2, i);
    int64_t p = (int64_t)((uint64_t)x * (uint64_t)y);  /* wrapping product */
    return p % n->m;                                    /* C99: truncated */
}

/* Evaluate the subtree rooted at nodes[*pos] for row i; *pos moves past it. */
static int eval_node(const otable *t, const onode *nodes, int32_t *pos, int64_t i)
{
    const onode *n = &nodes[(*pos)++];
    switch (n->kind) {
    case K_AND: {
        int r = 1;
        for (int32_t c = 0; c < n->nchild; ++c) r &= eval_node(t, nodes, pos, i);
        return r;
    }
    case K_OR: {
        int r = 0;
        for (int32_t c = 0; c < n->nchild; ++c) r |= eval_node(t, nodes, pos, i);
        return r;
    }
    case K_NOT:
        return !eval_node(t, nodes, pos, i);
    case K_CONST:
        return n->a != 0;
    case K_CMP: {
        int64_t x = operand_value(t, n, i);
        switch (n->op) {
        case OP_EQ: return x == n->a;
        case OP_NE: return x != n->a;
        case OP_LT: return x < n->a;
        case OP_LE: return x <= n->a;
        case OP_GT: return x > n->a;
        case OP_GE: return x >= n->a;
        }
        return 0;
    }
    case K_BETWEEN: {
        int64_t x = operand_value(t, n, i);
        int r = (n->a <= x) && (x <= n->b);
        return n->neg ? !r : r;
    }
    case K_IN: {
        int64_t x = operand_value(t, n, i);
        int r = 0;
        for (int32_t v = 0; v < n->nchild; ++v) r |= (x == t->vals[n->voff + v]);
        return n->neg ? !r : r;
    }
    }
    return 0;
}

/* Exact count of rows in [row0, row1) for which the predicate holds. */
int64_t oracle_count(const onode *nodes, const int64_t *vals, const void *const *cols,
                     const int32_t *dtypes, int64_t row0, int64_t row1)
{
    otable t = {cols, dtypes, vals};
    int64_t count = 0;
    for (int64_t i = row0; i < row1; ++i) {
        int32_t pos = 0;
        count += eval_node(&t, nodes, &pos, i);
    }
    return count;
}

/* Ascending ids of qualifying rows in [0, nrows); writes at most cap ids and
 * returns the full count. */
int64_t oracle_select(const onode *nodes, const int64_t *vals, const void *const *cols,
                      const int32_t *dtypes, int64_t nrows, uint32_t *ids, int64_t cap)
{
    otable t = {cols, dtypes, vals};
    int64_t count = 0;
    for (int64_t i = 0; i < nrows; ++i) {
        int32_t pos = 0;
        if (eval_node(&t, nodes, &pos, i)) {
            if (count < cap) ids[count] = (uint32_t)i;
            ++count;
        }
    }
    return count;
}

/* One byte per row: 1 when the predicate holds (the dense-key qualifying set). */
void oracle_mark(const onode *nodes, const int64_t *vals, const void *const *cols,
                 const int32_t *dtypes, int64_t nrows, uint8_t *mark)
{
    otable t = {cols, dtypes, vals};
    for (int64_t i = 0; i < nrows; ++i) {
        int32_t pos = 0;
        mark[i] = (uint8_t)eval_node(&t, nodes, &pos, i);
    }
}

/* Semi-join count for the dimension subset `subset` (bit d = dimension d),
 * rows [row0, row1) of the fact table.  marks[d][k] = 1 when dimension d's
 * row with dense key k qualifies. */
int64_t oracle_semijoin_count(const int32_t *const *fk, int32_t ndims,
                              const uint8_t *const *marks, const int64_t *dim_rows,
                              uint32_t subset, int64_t row0, int64_t row1)
{
    int64_t count = 0;
    for (int64_t i = row0; i < row1; ++i) {
        int ok = 1;
        for (int32_t d = 0; d < ndims; ++d) {
            if (!(subset >> d & 1u)) continue;
            int64_t k = fk[d][i];
            if (k < 0 || k >= dim_rows[d] || !marks[d][k]) { ok = 0; break; }
        }
        count += ok;
    }
    return count;
}
