"""Predicate text -> abstract syntax tree, for the oracle only.

Test infrastructure (see ``oracle/__init__.py``).  This parser is written
independently of the product library's compiler: the two share only the
predicate language, which mirrors the paper's selection sub-query (Sec. 1 and
Sec. 2: equality, BETWEEN, OR and a udf over several attributes of one table,
ANDed together).

Grammar (keywords case-insensitive)::

    pred    := or
    or      := and  ( OR and )*
    and     := unary ( AND unary )*
    unary   := NOT unary | atom
    atom    := '(' pred ')' | TRUE | FALSE | test
    test    := operand cmp INT
             | operand [NOT] BETWEEN INT AND INT
             | operand [NOT] IN '(' [ INT (',' INT)* ] ')'
    operand := IDENT | udf '(' IDENT ',' IDENT ',' INT ')'
    cmp     := '=' | '==' | '!=' | '<>' | '<' | '<=' | '>' | '>='

AST nodes are tuples:
    ('and', [c...]), ('or', [c...]), ('not', c), ('const', bool),
    ('cmp', op, operand, k), ('between', operand, lo, hi, negated),
    ('in', operand, [v...], negated);
    operand = ('col', name) | ('udf', name_a, name_b, m).
"""
from __future__ import annotations

import re
from typing import List, Tuple

_TOKEN = re.compile(r"\s*(?:(?P<int>-?\d+)|(?P<id>[A-Za-z_][A-Za-z0-9_]*)|"
                    r"(?P<op><=|>=|<>|!=|==|[=<>(),]))")
_KEYWORDS = {"AND", "OR", "NOT", "BETWEEN", "IN", "TRUE", "FALSE", "UDF"}


class OracleParseError(ValueError):
    pass


def _tokens(text: str) -> List[Tuple[str, str]]:
    out, pos = [], 0
    text = text.rstrip()
    while pos < len(text):
        m = _TOKEN.match(text, pos)
        if not m or m.end() == pos:
            raise OracleParseError(f"bad character at {pos}: {text[pos:pos + 10]!r}")
        pos = m.end()
        if m.group("int") is not None:
            out.append(("int", m.group("int")))
        elif m.group("id") is not None:
            w = m.group("id")
            out.append(("kw", w.upper()) if w.upper() in _KEYWORDS else ("id", w))
        else:
            out.append(("op", m.group("op")))
    out.append(("end", ""))
    return out


class _Parser:
    def __init__(self, text: str):
        self.t = _tokens(text)
        self.i = 0

    def peek(self):
        return self.t[self.i]

    def take(self, kind=None, val=None):
        k, v = self.t[self.i]
        if (kind is not None and k != kind) or (val is not None and v != val):
            raise OracleParseError(f"expected {val or kind}, got {v or k!r}")
        self.i += 1
        return v

    def integer(self) -> int:
        v = int(self.take("int"))
        if not -(1 << 63) <= v < (1 << 63):
            raise OracleParseError("integer constant outside int64")
        return v

    def pred(self):
        kids = [self.conj()]
        while self.peek() == ("kw", "OR"):
            self.take()
            kids.append(self.conj())
        return kids[0] if len(kids) == 1 else ("or", kids)

    def conj(self):
        kids = [self.unary()]
        while self.peek() == ("kw", "AND"):
            self.take()
            kids.append(self.unary())
        return kids[0] if len(kids) == 1 else ("and", kids)

    def unary(self):
        if self.peek() == ("kw", "NOT"):
            self.take()
            return ("not", self.unary())
        return self.atom()

    def atom(self):
        k, v = self.peek()
        if (k, v) == ("op", "("):
            self.take()
            e = self.pred()
            self.take("op", ")")
            return e
        if (k, v) == ("kw", "TRUE"):
            self.take()
            return ("const", True)
        if (k, v) == ("kw", "FALSE"):
            self.take()
            return ("const", False)
        return self.test()

    def operand(self):
        if self.peek() == ("kw", "UDF"):
            self.take()
            self.take("op", "(")
            a = self.take("id")
            self.take("op", ",")
            b = self.take("id")
            self.take("op", ",")
            m = self.integer()
            self.take("op", ")")
            if m <= 0:
                raise OracleParseError("udf modulus must be positive")
            return ("udf", a, b, m)
        return ("col", self.take("id"))

    def test(self):
        opd = self.operand()
        neg = False
        if self.peek() == ("kw", "NOT"):
            self.take()
            neg = True
        k, v = self.peek()
        if (k, v) == ("kw", "BETWEEN"):
            self.take()
            lo = self.integer()
            self.take("kw", "AND")
            hi = self.integer()
            return ("between", opd, lo, hi, neg)
        if (k, v) == ("kw", "IN"):
            self.take()
            self.take("op", "(")
            vals = []
            if self.peek() != ("op", ")"):
                vals.append(self.integer())
                while self.peek() == ("op", ","):
                    self.take()
                    vals.append(self.integer())
            self.take("op", ")")
            return ("in", opd, vals, neg)
        if neg:
            raise OracleParseError("NOT must precede BETWEEN or IN here")
        if k == "op" and v in ("=", "==", "!=", "<>", "<", "<=", ">", ">="):
            self.take()
            op = {"==": "=", "<>": "!="}.get(v, v)
            return ("cmp", op, opd, self.integer())
        raise OracleParseError(f"expected a comparison, got {v or k!r}")


def parse(text: str):
    p = _Parser(text)
    e = p.pred()
    p.take("end")
    return e


def columns_of(ast) -> List[str]:
    """Column names the predicate reads, in first-use order."""
    out: List[str] = []

    def opd(o):
        names = [o[1]] if o[0] == "col" else [o[1], o[2]]
        for n in names:
            if n not in out:
                out.append(n)

    def walk(e):
        k = e[0]
        if k in ("and", "or"):
            for c in e[1]:
                walk(c)
        elif k == "not":
            walk(e[1])
        elif k == "cmp":
            opd(e[2])
        elif k in ("between", "in"):
            opd(e[1])

    walk(ast)
    return out
