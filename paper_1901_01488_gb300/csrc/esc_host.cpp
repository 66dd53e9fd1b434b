// Host side of libesc: table registration, the predicate compiler and the
// error channel.  The compiler turns the WHERE clause of the selectivity
// sub-query (paper Sec. 1, Sec. 2) into a flat postfix program the scan
// kernel interprets on 8 rows per lane at a time.
//
// Lowering rules (all exact, integer):
//  * every comparison becomes an inclusive range on the operand, clamped to
//    the operand's value domain (u8 [0,255], u16 [0,65535], i32, i64, and
//    for udf(a,b,m) [-(m-1), m-1], or [0, m-1] when both columns are
//    unsigned); an empty range folds to FALSE, the full domain to TRUE;
//  * '!=' , NOT BETWEEN and NOT IN become NOT of the positive test;
//  * IN lists keep their in-domain distinct values; one value is a range;
//  * AND/OR are flattened and constant-folded, then emitted as binary chains
//    with the child that needs the deepest stack first (Sethi-Ullman order),
//    so the evaluation stack stays within 8 entries.
#include <algorithm>
#include <atomic>
#include <cctype>
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "esc_internal.h"

namespace esc {

static thread_local std::string g_err;

esc_status fail(esc_status s, const std::string &msg) {
  g_err = msg;
  return s;
}
void clear_error() { g_err.clear(); }

int dtype_width(int32_t dt) {
  switch (dt) {
    case ESC_I32: return 4;
    case ESC_I64: return 8;
    case ESC_U8: return 1;
    case ESC_U16: return 2;
  }
  return 0;
}

static const char *dtype_name(int32_t dt) {
  switch (dt) {
    case ESC_I32: return "i32";
    case ESC_I64: return "i64";
    case ESC_U8: return "u8";
    case ESC_U16: return "u16";
  }
  return "?";
}

static void dtype_domain(int32_t dt, int64_t *lo, int64_t *hi) {
  switch (dt) {
    case ESC_I32: *lo = INT32_MIN; *hi = INT32_MAX; return;
    case ESC_U8: *lo = 0; *hi = 255; return;
    case ESC_U16: *lo = 0; *hi = 65535; return;
    default: *lo = INT64_MIN; *hi = INT64_MAX; return;
  }
}

void udiv_magic(uint64_t d, uint64_t *mult, int32_t *sh1, int32_t *sh2) {
  // Granlund & Montgomery 1994, Fig. 4.1 (unsigned division, N = 64):
  // l = ceil(log2 d), m' = floor(2^N (2^l - d) / d) + 1,
  // sh1 = min(l, 1), sh2 = max(l - 1, 0).
  int l = 0;
  while (l < 64 && ((unsigned __int128)1 << l) < (unsigned __int128)d) ++l;
  unsigned __int128 two_l = (unsigned __int128)1 << l;
  unsigned __int128 num = (unsigned __int128)(uint64_t)(two_l - d) << 64;
  *mult = (uint64_t)(num / d) + 1;
  *sh1 = l < 1 ? l : 1;
  *sh2 = l - 1 > 0 ? l - 1 : 0;
}

// ------------------------------------------------------------------ parser
namespace {

struct Tok {
  enum Kind { INT, ID, KW, OP, END } kind;
  std::string s;
  int64_t v = 0;
  size_t pos = 0;
};

struct Ast {
  enum Kind { AND, OR, NOT, CONST, CMP, BETWEEN, IN } kind;
  std::vector<std::unique_ptr<Ast>> kids;
  bool value = false;      // CONST
  std::string op;          // CMP: = != < <= > >=
  bool neg = false;        // BETWEEN / IN
  bool udf = false;        // operand is udf(a, b, m)
  std::string a, b;        // operand column(s)
  int64_t m = 1;
  int64_t k = 0, lo = 0, hi = 0;
  std::vector<int64_t> vals;
};

struct ParseError {
  std::string msg;
};

class Parser {
 public:
  explicit Parser(const std::string &text) { lex(text); }

  std::unique_ptr<Ast> parse() {
    auto e = disj();
    if (t_[i_].kind != Tok::END) err("unexpected '" + t_[i_].s + "'");
    return e;
  }

 private:
  std::vector<Tok> t_;
  size_t i_ = 0;

  [[noreturn]] void err(const std::string &m) {
    throw ParseError{"predicate syntax error at offset " + std::to_string(t_[i_].pos) + ": " + m};
  }

  static bool is_kw(const std::string &u) {
    return u == "AND" || u == "OR" || u == "NOT" || u == "BETWEEN" || u == "IN" || u == "TRUE" ||
           u == "FALSE" || u == "UDF";
  }

  void lex(const std::string &s) {
    size_t p = 0;
    while (true) {
      while (p < s.size() && std::isspace((unsigned char)s[p])) ++p;
      Tok t;
      t.pos = p;
      if (p >= s.size()) {
        t.kind = Tok::END;
        t_.push_back(t);
        return;
      }
      char c = s[p];
      bool neg_int = c == '-' && p + 1 < s.size() && std::isdigit((unsigned char)s[p + 1]);
      if (std::isdigit((unsigned char)c) || neg_int) {
        size_t q = p + (neg_int ? 1 : 0);
        while (q < s.size() && std::isdigit((unsigned char)s[q])) ++q;
        std::string lit = s.substr(p, q - p);
        // exact int64 parse with overflow detection
        bool neg = lit[0] == '-';
        unsigned __int128 acc = 0;
        for (size_t k = neg ? 1 : 0; k < lit.size(); ++k) {
          acc = acc * 10 + (unsigned)(lit[k] - '0');
          if (acc > ((unsigned __int128)1 << 63)) break;
        }
        if ((!neg && acc > (unsigned __int128)INT64_MAX) || (neg && acc > ((unsigned __int128)1 << 63))) {
          i_ = t_.size();
          t_.push_back(t);
          t_.back().s = lit;
          err("integer constant outside int64: " + lit);
        }
        t.kind = Tok::INT;
        t.v = neg ? (int64_t)(0 - (uint64_t)acc) : (int64_t)acc;
        t.s = lit;
        p = q;
      } else if (std::isalpha((unsigned char)c) || c == '_') {
        size_t q = p;
        while (q < s.size() && (std::isalnum((unsigned char)s[q]) || s[q] == '_')) ++q;
        t.s = s.substr(p, q - p);
        std::string u = t.s;
        for (auto &ch : u) ch = (char)std::toupper((unsigned char)ch);
        if (is_kw(u)) {
          t.kind = Tok::KW;
          t.s = u;
        } else {
          t.kind = Tok::ID;
        }
        p = q;
      } else {
        static const char *two[] = {"<=", ">=", "<>", "!=", "=="};
        t.kind = Tok::OP;
        bool done = false;
        for (const char *o : two) {
          if (s.compare(p, 2, o) == 0) {
            t.s = o;
            p += 2;
            done = true;
            break;
          }
        }
        if (!done) {
          if (std::strchr("=<>(),", c) == nullptr) {
            i_ = t_.size();
            t.s = std::string(1, c);
            t_.push_back(t);
            err(std::string("unexpected character '") + c + "'");
          }
          t.s = std::string(1, c);
          ++p;
        }
      }
      t_.push_back(t);
    }
  }

  bool at(Tok::Kind k, const char *s = nullptr) const {
    return t_[i_].kind == k && (s == nullptr || t_[i_].s == s);
  }
  Tok take(Tok::Kind k, const char *s = nullptr) {
    if (!at(k, s)) err(std::string("expected ") + (s ? s : "token") + ", got '" + t_[i_].s + "'");
    return t_[i_++];
  }

  std::unique_ptr<Ast> disj() {
    auto first = conj();
    if (!at(Tok::KW, "OR")) return first;
    auto n = std::make_unique<Ast>();
    n->kind = Ast::OR;
    n->kids.push_back(std::move(first));
    while (at(Tok::KW, "OR")) {
      ++i_;
      n->kids.push_back(conj());
    }
    return n;
  }

  std::unique_ptr<Ast> conj() {
    auto first = unary();
    if (!at(Tok::KW, "AND")) return first;
    auto n = std::make_unique<Ast>();
    n->kind = Ast::AND;
    n->kids.push_back(std::move(first));
    while (at(Tok::KW, "AND")) {
      ++i_;
      n->kids.push_back(unary());
    }
    return n;
  }

  std::unique_ptr<Ast> unary() {
    if (at(Tok::KW, "NOT")) {
      ++i_;
      auto n = std::make_unique<Ast>();
      n->kind = Ast::NOT;
      n->kids.push_back(unary());
      return n;
    }
    if (at(Tok::OP, "(")) {
      ++i_;
      auto e = disj();
      take(Tok::OP, ")");
      return e;
    }
    if (at(Tok::KW, "TRUE") || at(Tok::KW, "FALSE")) {
      auto n = std::make_unique<Ast>();
      n->kind = Ast::CONST;
      n->value = t_[i_].s == "TRUE";
      ++i_;
      return n;
    }
    return test();
  }

  std::unique_ptr<Ast> test() {
    auto n = std::make_unique<Ast>();
    if (at(Tok::KW, "UDF")) {
      ++i_;
      take(Tok::OP, "(");
      n->udf = true;
      n->a = take(Tok::ID).s;
      take(Tok::OP, ",");
      n->b = take(Tok::ID).s;
      take(Tok::OP, ",");
      n->m = take(Tok::INT).v;
      take(Tok::OP, ")");
      if (n->m <= 0) err("udf modulus must be positive");
    } else {
      n->a = take(Tok::ID).s;
    }
    bool neg = false;
    if (at(Tok::KW, "NOT")) {
      ++i_;
      neg = true;
    }
    if (at(Tok::KW, "BETWEEN")) {
      ++i_;
      n->kind = Ast::BETWEEN;
      n->neg = neg;
      n->lo = take(Tok::INT).v;
      take(Tok::KW, "AND");
      n->hi = take(Tok::INT).v;
      return n;
    }
    if (at(Tok::KW, "IN")) {
      ++i_;
      n->kind = Ast::IN;
      n->neg = neg;
      take(Tok::OP, "(");
      if (!at(Tok::OP, ")")) {
        n->vals.push_back(take(Tok::INT).v);
        while (at(Tok::OP, ",")) {
          ++i_;
          n->vals.push_back(take(Tok::INT).v);
        }
      }
      take(Tok::OP, ")");
      if ((int)n->vals.size() > kMaxIn) err("IN list longer than 16 values");
      return n;
    }
    if (neg) err("NOT must be followed by BETWEEN or IN here");
    if (t_[i_].kind == Tok::OP) {
      std::string op = t_[i_].s;
      if (op == "==") op = "=";
      if (op == "<>") op = "!=";
      if (op == "=" || op == "!=" || op == "<" || op == "<=" || op == ">" || op == ">=") {
        ++i_;
        n->kind = Ast::CMP;
        n->op = op;
        n->k = take(Tok::INT).v;
        return n;
      }
    }
    err("expected a comparison after the operand");
  }
};

// ------------------------------------------------------------------ lowering
struct Low {
  enum Kind { AND, OR, NOT, TRUE_, FALSE_, LEAF } kind;
  std::vector<Low> kids;
  Instr leaf{};                 // op RANGE / IN / UDF with column *table* indices in ref/ref2
  int col = -1, col2 = -1;      // table column indices
  int64_t m = 1;                // udf modulus
  std::vector<int64_t> vals;    // IN values
};

Low mk(Low::Kind k) {
  Low l;
  l.kind = k;
  return l;
}

Low negate(Low x) {
  if (x.kind == Low::TRUE_) return mk(Low::FALSE_);
  if (x.kind == Low::FALSE_) return mk(Low::TRUE_);
  if (x.kind == Low::NOT) return std::move(x.kids[0]);
  Low n = mk(Low::NOT);
  n.kids.push_back(std::move(x));
  return n;
}

struct Lowerer {
  const esc_table *t;

  int column(const std::string &name) {
    for (size_t i = 0; i < t->names.size(); ++i)
      if (t->names[i] == name) return (int)i;
    throw ParseError{"unknown column '" + name + "'"};
  }

  // Positive range test on an operand, clamped to its domain.
  Low range(const Ast &a, int64_t lo, int64_t hi) {
    int64_t dlo, dhi;
    Low leaf = mk(Low::LEAF);
    leaf.col = column(a.a);
    if (a.udf) {
      leaf.col2 = column(a.b);
      leaf.m = a.m;
      bool uns = (t->dtypes[leaf.col] == ESC_U8 || t->dtypes[leaf.col] == ESC_U16) &&
                 (t->dtypes[leaf.col2] == ESC_U8 || t->dtypes[leaf.col2] == ESC_U16);
      dhi = a.m - 1;
      dlo = uns ? 0 : -(a.m - 1);
      leaf.leaf.op = OP_UDF;
    } else {
      dtype_domain(t->dtypes[leaf.col], &dlo, &dhi);
      leaf.leaf.op = OP_RANGE;
    }
    lo = std::max(lo, dlo);
    hi = std::min(hi, dhi);
    if (lo > hi) return mk(Low::FALSE_);
    if (lo == dlo && hi == dhi) return mk(Low::TRUE_);
    leaf.leaf.lo = lo;
    leaf.leaf.hi = hi;
    return leaf;
  }

  bool udf_unsigned(int col, int col2) const {
    auto u = [&](int c) { return t->dtypes[c] == ESC_U8 || t->dtypes[c] == ESC_U16; };
    return u(col) && u(col2);
  }

  // Value domain of a leaf's operand.
  void domain(const Low &l, int64_t *dlo, int64_t *dhi) const {
    if (l.leaf.op == OP_UDF) {
      *dhi = l.m - 1;
      *dlo = udf_unsigned(l.col, l.col2) ? 0 : -(l.m - 1);
    } else {
      dtype_domain(t->dtypes[l.col], dlo, dhi);
    }
  }

  // Key of a leaf's operand: a column, or udf(a, b, m) with {a, b} unordered
  // (the wrapped product commutes).  Empty for anything else.
  static std::string operand_key(const Low &l) {
    if (l.kind != Low::LEAF) return std::string();
    if (l.leaf.op == OP_UDF)
      return "u" + std::to_string(std::min(l.col, l.col2)) + "," + std::to_string(std::max(l.col, l.col2)) + "," +
             std::to_string(l.m);
    return "c" + std::to_string(l.col);
  }

  // Tests on the same operand among the children of one AND (is_and) or OR
  // combine into at most one range and one IN list for that operand:
  //  * AND: ranges intersect; IN lists intersect and keep only values inside
  //    the range, which the list then replaces; an empty result makes the
  //    whole AND false (returns false);
  //  * OR: overlapping or adjacent ranges unite; IN lists unite and lose the
  //    values some range already holds; a range covering the operand's
  //    domain makes the whole OR true (returns false).
  // Exact set algebra on integers, so results never change.
  bool merge_same_operand(std::vector<Low> &kids, bool is_and) {
    std::vector<Low> out;
    std::vector<std::string> keys;
    std::vector<std::vector<size_t>> groups;
    for (size_t i = 0; i < kids.size(); ++i) {
      const std::string k = operand_key(kids[i]);
      size_t g = keys.size();
      if (!k.empty())
        for (size_t j = 0; j < keys.size(); ++j)
          if (keys[j] == k) g = j;
      if (g == keys.size()) {
        keys.push_back(k);
        groups.emplace_back();
      }
      groups[g].push_back(i);
    }
    for (size_t g = 0; g < groups.size(); ++g) {
      if (keys[g].empty() || groups[g].size() == 1) {
        for (size_t i : groups[g]) out.push_back(std::move(kids[i]));
        continue;
      }
      const Low &proto = kids[groups[g][0]];
      int64_t dlo, dhi;
      domain(proto, &dlo, &dhi);
      std::vector<std::pair<int64_t, int64_t>> ranges;
      std::vector<std::set<int64_t>> lists;
      for (size_t i : groups[g]) {
        const Low &l = kids[i];
        if (l.leaf.op == OP_IN) lists.emplace_back(l.vals.begin(), l.vals.end());
        else ranges.push_back({l.leaf.lo, l.leaf.hi});
      }
      std::vector<std::pair<int64_t, int64_t>> rs;
      std::set<int64_t> vals;
      bool have_list = !lists.empty();
      if (is_and) {
        if (!ranges.empty()) {
          int64_t lo = INT64_MIN, hi = INT64_MAX;
          for (auto &r : ranges) {
            lo = std::max(lo, r.first);
            hi = std::min(hi, r.second);
          }
          if (lo > hi) return false;
          rs.push_back({lo, hi});
        }
        if (have_list) {
          vals = lists[0];
          for (size_t k = 1; k < lists.size(); ++k) {
            std::set<int64_t> both;
            for (int64_t v : vals)
              if (lists[k].count(v)) both.insert(v);
            vals.swap(both);
          }
          if (!rs.empty()) {
            std::set<int64_t> in;
            for (int64_t v : vals)
              if (v >= rs[0].first && v <= rs[0].second) in.insert(v);
            vals.swap(in);
            rs.clear();  // every value left is inside the range
          }
          if (vals.empty()) return false;
        }
      } else {
        std::sort(ranges.begin(), ranges.end());
        for (auto &r : ranges) {
          if (!rs.empty() && (rs.back().second == INT64_MAX || rs.back().second + 1 >= r.first))
            rs.back().second = std::max(rs.back().second, r.second);
          else
            rs.push_back(r);
        }
        for (auto &r : rs)
          if (r.first <= dlo && r.second >= dhi) return false;
        for (auto &l : lists)
          for (int64_t v : l) {
            bool held = false;
            for (auto &r : rs) held = held || (v >= r.first && v <= r.second);
            if (!held) vals.insert(v);
          }
        have_list = !vals.empty();
      }
      for (auto &r : rs) {
        Low leaf = proto;
        leaf.vals.clear();
        leaf.leaf.op = proto.leaf.op == OP_UDF ? OP_UDF : OP_RANGE;
        leaf.leaf.lo = r.first;
        leaf.leaf.hi = r.second;
        out.push_back(std::move(leaf));
      }
      if (have_list) {
        Low leaf = proto;
        if (vals.size() == 1) {
          leaf.vals.clear();
          leaf.leaf.op = OP_RANGE;
          leaf.leaf.lo = leaf.leaf.hi = *vals.begin();
        } else {
          leaf.leaf.op = OP_IN;
          leaf.leaf.lo = leaf.leaf.hi = 0;
          leaf.vals.assign(vals.begin(), vals.end());
        }
        out.push_back(std::move(leaf));
      }
    }
    kids = std::move(out);
    return true;
  }

  Low lower(const Ast &a) {
    switch (a.kind) {
      case Ast::CONST: return mk(a.value ? Low::TRUE_ : Low::FALSE_);
      case Ast::NOT: return negate(lower(*a.kids[0]));
      case Ast::CMP: {
        const int64_t k = a.k;
        if (a.op == "=") return range(a, k, k);
        if (a.op == "!=") return negate(range(a, k, k));
        if (a.op == "<") return k == INT64_MIN ? (column(a.a), mk(Low::FALSE_)) : range(a, INT64_MIN, k - 1);
        if (a.op == "<=") return range(a, INT64_MIN, k);
        if (a.op == ">") return k == INT64_MAX ? (column(a.a), mk(Low::FALSE_)) : range(a, k + 1, INT64_MAX);
        return range(a, k, INT64_MAX);  // >=
      }
      case Ast::BETWEEN: {
        Low r = a.lo > a.hi ? (column(a.a), mk(Low::FALSE_)) : range(a, a.lo, a.hi);
        return a.neg ? negate(std::move(r)) : r;
      }
      case Ast::IN: {
        // keep distinct values inside the operand's domain
        Low probe = range(a, INT64_MIN, INT64_MAX);  // resolves columns; TRUE_ (full domain)
        (void)probe;
        int64_t dlo, dhi;
        int col = column(a.a);
        if (a.udf) {
          int col2 = column(a.b);
          bool uns = (t->dtypes[col] == ESC_U8 || t->dtypes[col] == ESC_U16) &&
                     (t->dtypes[col2] == ESC_U8 || t->dtypes[col2] == ESC_U16);
          dhi = a.m - 1;
          dlo = uns ? 0 : -(a.m - 1);
        } else {
          dtype_domain(t->dtypes[col], &dlo, &dhi);
        }
        std::set<int64_t> vs;
        for (int64_t v : a.vals)
          if (v >= dlo && v <= dhi) vs.insert(v);
        Low r;
        if (vs.empty()) {
          r = mk(Low::FALSE_);
        } else if (vs.size() == 1 || a.udf) {
          // a udf IN list is an OR of point ranges on the udf value
          Low o = mk(Low::OR);
          for (int64_t v : vs) o.kids.push_back(range(a, v, v));
          r = o.kids.size() == 1 ? std::move(o.kids[0]) : std::move(o);
        } else {
          r = mk(Low::LEAF);
          r.col = col;
          r.leaf.op = OP_IN;
          r.vals.assign(vs.begin(), vs.end());
        }
        return a.neg ? negate(std::move(r)) : r;
      }
      case Ast::AND:
      case Ast::OR: {
        const bool is_and = a.kind == Ast::AND;
        Low n = mk(is_and ? Low::AND : Low::OR);
        for (auto &k : a.kids) {
          Low c = lower(*k);
          if (c.kind == (is_and ? Low::TRUE_ : Low::FALSE_)) continue;           // identity
          if (c.kind == (is_and ? Low::FALSE_ : Low::TRUE_)) return c;           // absorbing
          if (c.kind == n.kind) {                                                // flatten
            for (auto &g : c.kids) n.kids.push_back(std::move(g));
          } else {
            n.kids.push_back(std::move(c));
          }
        }
        // tests on one operand combine: AND intersects, OR unites
        if (!merge_same_operand(n.kids, is_and)) return mk(is_and ? Low::FALSE_ : Low::TRUE_);
        if (n.kids.empty()) return mk(is_and ? Low::TRUE_ : Low::FALSE_);
        if (n.kids.size() == 1) return std::move(n.kids[0]);
        return n;
      }
    }
    throw ParseError{"internal: bad node"};
  }
};

// Rough evaluation cost of a subtree in units of one 32-bit range test.
double cost(const Low &l) {
  switch (l.kind) {
    case Low::LEAF:
      if (l.leaf.op == OP_UDF) return 6.0;
      if (l.leaf.op == OP_IN) {
        bool small = true;
        for (int64_t v : l.vals) small = small && v >= 0 && v < 256;
        return small ? 1.5 : 1.0 + 0.25 * (double)l.vals.size();
      }
      return 1.0;  // range
    case Low::NOT: return cost(l.kids[0]);
    case Low::AND:
    case Low::OR: {
      double c = 0;
      for (auto &k : l.kids) c += cost(k) + 0.2;
      return c;
    }
    default: return 0.1;
  }
}

int need(const Low &l) {
  switch (l.kind) {
    case Low::NOT: return need(l.kids[0]);
    case Low::AND:
    case Low::OR: {
      std::vector<int> d;
      for (auto &k : l.kids) d.push_back(need(k));
      std::sort(d.rbegin(), d.rend());
      int m = 0;
      for (size_t i = 0; i < d.size(); ++i) m = std::max(m, d[i] + (i > 0 ? 1 : 0));
      return m;
    }
    default: return 1;
  }
}

struct Emitter {
  esc_pred *p;
  std::vector<int> slot_of_col;
  bool su_only = false;  // order every AND/OR deepest first

  int slot(int col) {
    if (slot_of_col[col] < 0) {
      if ((int)p->ref_cols.size() >= kMaxRef) throw ParseError{"predicate reads more than 16 columns"};
      slot_of_col[col] = (int)p->ref_cols.size();
      p->ref_cols.push_back(col);
    }
    return slot_of_col[col];
  }

  void push(const Instr &ins) {
    if ((int)p->code.size() >= kMaxInstr) throw ParseError{"predicate needs more than 64 instructions"};
    p->code.push_back(ins);
  }

  int pool(int64_t v) {
    if ((int)p->pool.size() >= kMaxPool) throw ParseError{"predicate constants exceed the 128-entry pool"};
    p->pool.push_back(v);
    return (int)p->pool.size() - 1;
  }

  void emit(const Low &l) {
    Instr ins{};
    switch (l.kind) {
      case Low::TRUE_: ins.op = OP_TRUE; push(ins); return;
      case Low::FALSE_: ins.op = OP_FALSE; push(ins); return;
      case Low::NOT:
        emit(l.kids[0]);
        ins.op = OP_NOT;
        push(ins);
        return;
      case Low::AND:
      case Low::OR: {
        // Children cheapest first, so that a cheap test decides as many rows as
        // possible before the costly ones run; if that order would need more
        // than kMaxDepth stack entries, deepest first (Sethi-Ullman).  Before
        // each later child that is costly enough, a conditional jump skips it
        // and the combining op when the result so far already decides the
        // connective for all rows a warp holds.
        std::vector<std::pair<double, size_t>> order;
        for (size_t i = 0; i < l.kids.size(); ++i) order.push_back({cost(l.kids[i]), i});
        std::stable_sort(order.begin(), order.end());
        int depth = 0;
        for (size_t j = 0; j < order.size(); ++j)
          depth = std::max(depth, need(l.kids[order[j].second]) + (j > 0 ? 1 : 0));
        if (su_only || depth > kMaxDepth) {
          order.clear();
          for (size_t i = 0; i < l.kids.size(); ++i) order.push_back({(double)-need(l.kids[i]), i});
          std::stable_sort(order.begin(), order.end());
        }
        for (size_t j = 0; j < order.size(); ++j) {
          size_t jump = 0;
          const bool skippable = j > 0 && cost(l.kids[order[j].second]) >= 2.0;
          if (skippable) {
            Instr jz{};
            jz.op = l.kind == Low::AND ? OP_JZ : OP_JNZ;
            jump = p->code.size();
            push(jz);
          }
          emit(l.kids[order[j].second]);
          if (j > 0) {
            Instr c{};
            c.op = l.kind == Low::AND ? OP_AND : OP_OR;
            push(c);
            if (skippable) p->code[jump].off = (uint16_t)p->code.size();
          }
        }
        return;
      }
      case Low::LEAF: {
        ins = l.leaf;
        ins.dtype = (uint8_t)p->table->dtypes[l.col];
        ins.ref = (uint8_t)slot(l.col);
        if (ins.op == OP_UDF) {
          ins.dtype2 = (uint8_t)p->table->dtypes[l.col2];
          ins.ref2 = (uint8_t)slot(l.col2);
          uint64_t mult;
          int32_t s1, s2;
          udiv_magic((uint64_t)l.m, &mult, &s1, &s2);
          ins.off = (uint16_t)pool(l.m);
          pool((int64_t)mult);
          pool((int64_t)s1);
          pool((int64_t)s2);
          // moduli below 2^16: ceil(2^64 / m) for Lemire, Kaser & Kurz's direct
          // 32-bit remainder (Softw. Pract. Exper. 2019), and 2^32 mod m
          const uint64_t um = (uint64_t)l.m;
          pool(um < 65536 ? (int64_t)(~0ull / um + 1) : 0);
          pool(um < 65536 ? (int64_t)((1ull << 32) % um) : 0);
        } else if (ins.op == OP_IN && !l.vals.empty() &&
                   (uint64_t)l.vals.back() - (uint64_t)l.vals.front() == (uint64_t)(l.vals.size() - 1)) {
          // the values (sorted, distinct) are one run of consecutive integers:
          // a single range test, cheaper than a set lookup
          ins.op = OP_RANGE;
          ins.lo = l.vals.front();
          ins.hi = l.vals.back();
          ins.n = 0;
        } else if (ins.op == OP_IN) {
          ins.n = (uint16_t)l.vals.size();
          bool small = true;
          for (int64_t v : l.vals) small = small && v >= 0 && v < 256;
          if (small) {
            // 256-bit membership set: bit v of word v / 32, two words per pool entry
            uint32_t words[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int64_t v : l.vals) words[v >> 5] |= 1u << (v & 31);
            ins.op = OP_INSET;
            ins.off = (uint16_t)p->pool.size();
            for (int k = 0; k < 4; ++k) pool((int64_t)(((uint64_t)words[2 * k + 1] << 32) | words[2 * k]));
            // the values themselves follow, for the program listing
            ins.lo = (int64_t)p->pool.size();
            for (int64_t v : l.vals) pool(v);
          } else {
            ins.off = (uint16_t)p->pool.size();
            for (int64_t v : l.vals) pool(v);
          }
        }
        push(ins);
        return;
      }
    }
  }
};

// Largest evaluation-stack depth the program reaches (jumps never skip a push
// without its matching pop, so straight-line simulation is exact).
int stack_depth(const std::vector<Instr> &code) {
  int d = 0, m = 0;
  for (const Instr &I : code) {
    switch (I.op) {
      case OP_AND:
      case OP_OR: --d; break;
      case OP_NOT:
      case OP_JZ:
      case OP_JNZ: break;
      default: m = std::max(m, ++d); break;
    }
  }
  return m;
}

}  // namespace

void fill_query_program(const esc_pred *p, Query *q) {
  q->ninstr = p->ninstr;
  q->nref = (int32_t)p->ref_cols.size();
  q->nproj = (int32_t)p->proj_cols.size();
  for (int i = 0; i < q->nref; ++i) {
    int c = p->ref_cols[i];
    q->ref_w[i] = (uint8_t)dtype_width(p->table->dtypes[c]);
    q->ref_ptr[i] = (const uint8_t *)p->table->data[c];
  }
  for (int i = 0; i < q->nproj; ++i) {
    int c = p->proj_cols[i];
    q->proj_w[i] = (uint8_t)dtype_width(p->table->dtypes[c]);
    q->proj_ptr[i] = (const uint8_t *)p->table->data[c];
    q->proj_ref[i] = (int8_t)p->proj_ref[i];
  }
  for (int i = 0; i < p->ninstr; ++i) q->code[i] = p->code[i];
  for (size_t i = 0; i < p->pool.size(); ++i) q->pool[i] = p->pool[i];
}

std::atomic<int32_t> g_fail_allocs{0};

bool inject_alloc_failure() {
  int32_t n = g_fail_allocs.load();
  while (n > 0 && !g_fail_allocs.compare_exchange_weak(n, n - 1)) {
  }
  return n > 0;
}

esc_status device_status(const ScratchHdr &h, const char *where) {
  if (h.status == (unsigned)ESC_EBOUNDS)
    return fail(ESC_EBOUNDS, std::string(where) + ": checked build: an index out of range at site " +
                                 std::to_string(h.site) + " (" + std::to_string(h.value) + "), access skipped");
  return fail((esc_status)h.status, std::string(where) + ": a bounded device-side wait gave up");
}

// Compaction-unit layout of a materialising call (defined with the kernels).
void layout_write_units(Query &q, int slots);

}  // namespace esc

using namespace esc;

// ------------------------------------------------------------------ C ABI
extern "C" {

const char *esc_last_error(void) { return g_err.c_str(); }

const char *esc_status_string(esc_status s) {
  switch (s) {
    case ESC_OK: return "ESC_OK";
    case ESC_EINVAL: return "ESC_EINVAL";
    case ESC_ETYPE: return "ESC_ETYPE";
    case ESC_ENOMEM: return "ESC_ENOMEM";
    case ESC_ETRUNC: return "ESC_ETRUNC";
    case ESC_ETIMEOUT: return "ESC_ETIMEOUT";
    case ESC_EBUSY: return "ESC_EBUSY";
    case ESC_ECUDA: return "ESC_ECUDA";
    case ESC_EBOUNDS: return "ESC_EBOUNDS";
  }
  return "ESC_UNKNOWN";
}

esc_status esc_debug_fail_allocs(int32_t n) {
  if (n < 0) return fail(ESC_EINVAL, "esc_debug_fail_allocs: n must be >= 0");
  g_fail_allocs.store(n);
  clear_error();
  return ESC_OK;
}

esc_status esc_debug_write_units(uint64_t nrows, int32_t slots, uint32_t *out) {
  if (!out || nrows > ESC_MAX_ROWS || slots < 0) return fail(ESC_EINVAL, "esc_debug_write_units: bad argument");
  esc::Query q;
  std::memset(&q, 0, sizeof q);
  q.nrows = (uint32_t)nrows;
  esc::layout_write_units(q, slots);
  out[0] = q.wunit_groups;
  out[1] = q.nwunits;
  out[2] = q.wunit_recip;
  clear_error();
  return ESC_OK;
}

esc_status esc_build_checked(int32_t *flag) {
  if (!flag) return fail(ESC_EINVAL, "esc_build_checked: flag is NULL");
#ifdef ESC_CHECKED
  *flag = 1;
#else
  *flag = 0;
#endif
  return ESC_OK;
}

esc_status esc_udf_magic(uint64_t d, uint64_t *mult, int32_t *sh1, int32_t *sh2) {
  if (d == 0 || !mult || !sh1 || !sh2) return fail(ESC_EINVAL, "esc_udf_magic: d must be >= 1");
  udiv_magic(d, mult, sh1, sh2);
  return ESC_OK;
}

esc_status esc_table_create(const esc_column *cols, int32_t ncols, uint64_t nrows, esc_table **out) {
  if (!out) return fail(ESC_EINVAL, "esc_table_create: out is NULL");
  *out = nullptr;
  if (!cols || ncols < 1 || ncols > 64) return fail(ESC_EINVAL, "esc_table_create: need 1..64 columns");
  if (nrows > ESC_MAX_ROWS) return fail(ESC_EINVAL, "esc_table_create: nrows must be at most 2^32 - 2^16");
  std::unique_ptr<esc_table> t(new (std::nothrow) esc_table);
  if (!t) return fail(ESC_ENOMEM, "esc_table_create: out of host memory");
  t->nrows = nrows;
  for (int i = 0; i < ncols; ++i) {
    const esc_column &c = cols[i];
    if (!c.name || !*c.name) return fail(ESC_EINVAL, "esc_table_create: column without a name");
    std::string nm(c.name);
    bool ident = std::isalpha((unsigned char)nm[0]) || nm[0] == '_';
    for (char ch : nm) ident = ident && (std::isalnum((unsigned char)ch) || ch == '_');
    if (!ident) return fail(ESC_EINVAL, "esc_table_create: column name '" + nm + "' is not an identifier");
    for (auto &o : t->names)
      if (o == nm) return fail(ESC_EINVAL, "esc_table_create: duplicate column name '" + nm + "'");
    if (dtype_width(c.dtype) == 0) return fail(ESC_ETYPE, "esc_table_create: column '" + nm + "' has an unknown dtype");
    if (nrows > 0 && !c.data) return fail(ESC_EINVAL, "esc_table_create: column '" + nm + "' has no data");
    if (((uintptr_t)c.data & 15u) != 0)
      return fail(ESC_EINVAL, "esc_table_create: column '" + nm + "' is not 16-byte aligned");
    t->names.push_back(nm);
    t->dtypes.push_back(c.dtype);
    t->data.push_back(c.data);
  }
  *out = t.release();
  clear_error();
  return ESC_OK;
}

esc_status esc_table_destroy(esc_table *t) {
  delete t;
  return ESC_OK;
}

uint64_t esc_table_nrows(const esc_table *t) { return t ? t->nrows : 0; }

esc_status esc_predicate_compile(const esc_table *t, const char *text, const char *const *proj,
                                 int32_t nproj, esc_pred **out) {
  ESC_RANGE("esc_predicate_compile");
  if (!out) return fail(ESC_EINVAL, "esc_predicate_compile: out is NULL");
  *out = nullptr;
  if (!t || !text) return fail(ESC_EINVAL, "esc_predicate_compile: table and text are required");
  if (nproj < 0 || nproj > kMaxProj || (nproj > 0 && !proj))
    return fail(ESC_EINVAL, "esc_predicate_compile: 0..16 projected columns");
  std::unique_ptr<esc_pred> p(new (std::nothrow) esc_pred);
  if (!p) return fail(ESC_ENOMEM, "esc_predicate_compile: out of host memory");
  p->table = t;
  p->text = text;
  try {
    Parser parser{std::string(text)};
    auto ast = parser.parse();
    Lowerer lw{t};
    Low low = lw.lower(*ast);
    if (need(low) > kMaxDepth) throw ParseError{"predicate nests too deeply (needs more than 8 stack entries)"};
    Emitter em{p.get(), std::vector<int>(t->names.size(), -1)};
    em.emit(low);
    p->depth = stack_depth(p->code);
    if (p->depth > kMaxDepth) {  // the cheapest-first order went too deep: deepest first everywhere
      p->code.clear();
      p->pool.clear();
      p->ref_cols.clear();
      em = Emitter{p.get(), std::vector<int>(t->names.size(), -1)};
      em.su_only = true;
      em.emit(low);
      p->depth = stack_depth(p->code);
    }
    p->ninstr = (int32_t)p->code.size();
    for (int i = 0; i < nproj; ++i) {
      if (!proj[i]) throw ParseError{"projected column name is NULL"};
      int c = lw.column(proj[i]);
      p->proj_cols.push_back(c);
      p->proj_ref.push_back(em.slot_of_col[c]);
    }
  } catch (const ParseError &e) {
    return fail(ESC_EINVAL, "esc_predicate_compile: " + e.msg);
  } catch (const std::bad_alloc &) {
    return fail(ESC_ENOMEM, "esc_predicate_compile: out of host memory");
  }
  *out = p.release();
  clear_error();
  return ESC_OK;
}

esc_status esc_predicate_set_tuning(esc_pred *p, const esc_tuning *t) {
  if (!p) return fail(ESC_EINVAL, "esc_predicate_set_tuning: pred is NULL");
  if (!t) {
    p->tuning = kDefaultTuning;
    return ESC_OK;
  }
  if (t->max_tile_rows < 256 || t->max_tile_rows > 32768 || t->max_tile_rows % 256 != 0)
    return fail(ESC_EINVAL, "esc_predicate_set_tuning: max_tile_rows must be a multiple of 256 in 256..32768");
  if (t->max_unit_kb < 16 || t->max_unit_kb > 4096)
    return fail(ESC_EINVAL, "esc_predicate_set_tuning: max_unit_kb must be in 16..4096");
  if (t->units_per_sm < 1 || t->units_per_sm > 64)
    return fail(ESC_EINVAL, "esc_predicate_set_tuning: units_per_sm must be in 1..64");
  bool udf = false;
  for (const Instr &I : p->code) udf = udf || I.op == OP_UDF;
  if (scan_shape_for(t->consumer_warps, t->rows_per_pass, udf, 0) < 0)
    return fail(ESC_EINVAL, "esc_predicate_set_tuning: no compiled scan shape has " + std::to_string(t->consumer_warps) +
                                " consumer warps and " + std::to_string(t->rows_per_pass) + " rows per pass" +
                                (udf ? " with the udf path" : ""));
  p->tuning = *t;
  clear_error();
  return ESC_OK;
}

esc_status esc_predicate_get_tuning(const esc_pred *p, esc_tuning *out) {
  if (!p || !out) return fail(ESC_EINVAL, "esc_predicate_get_tuning: NULL argument");
  *out = p->tuning;
  return ESC_OK;
}

esc_status esc_predicate_destroy(esc_pred *p) {
  delete p;
  return ESC_OK;
}

esc_status esc_predicate_compile_many(const esc_table *t, const char *const *texts, int32_t n,
                                      const char *const *proj, int32_t nproj, esc_pred **out, int32_t nthreads) {
  ESC_RANGE("esc_predicate_compile_many");
  if (n < 0 || (n > 0 && (!texts || !out)))
    return fail(ESC_EINVAL, "esc_predicate_compile_many: bad arguments");
  for (int32_t i = 0; i < n; ++i) out[i] = nullptr;
  if (n == 0) {
    clear_error();
    return ESC_OK;
  }
  // contiguous ranges of at least 64 predicates per thread; the compiler has
  // no shared mutable state (its error message is per thread)
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  int nt = nthreads > 0 ? nthreads : hw;
  nt = std::max(1, std::min({nt, 64, std::max(1, (int)(n / 64))}));
  std::vector<esc_status> st((size_t)nt, ESC_OK);
  std::vector<int32_t> bad((size_t)nt, -1);
  std::vector<std::string> msg((size_t)nt);
  auto work = [&](int k) {
    const int32_t i0 = (int32_t)((int64_t)n * k / nt), i1 = (int32_t)((int64_t)n * (k + 1) / nt);
    for (int32_t i = i0; i < i1; ++i) {
      const esc_status s = esc_predicate_compile(t, texts[i], proj, nproj, &out[i]);
      if (s != ESC_OK) {
        st[(size_t)k] = s;
        bad[(size_t)k] = i;
        msg[(size_t)k] = esc_last_error();
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  int started = 1;
  try {
    for (; started < nt; ++started) pool.emplace_back(work, started);
  } catch (...) {  // no more threads: the rest of the ranges run here
  }
  work(0);
  for (int k = started; k < nt; ++k) work(k);
  for (auto &th : pool) th.join();
  for (int k = 0; k < nt; ++k) {
    if (st[(size_t)k] == ESC_OK) continue;
    for (int32_t i = 0; i < n; ++i) {
      delete out[i];
      out[i] = nullptr;
    }
    return fail(st[(size_t)k], "esc_predicate_compile_many: predicate " + std::to_string(bad[(size_t)k]) + ": " +
                                   msg[(size_t)k]);
  }
  clear_error();
  return ESC_OK;
}

esc_status esc_predicate_explain(const esc_pred *p, char *buf, uint64_t buflen) {
  if (!p || !buf || buflen == 0) return fail(ESC_EINVAL, "esc_predicate_explain: bad arguments");
  std::string s;
  char line[512];
  const esc_table *t = p->table;
  std::snprintf(line, sizeof line, "rows %" PRIu64 "\ndepth %d\n", t->nrows, p->depth);
  s += line;
  for (size_t i = 0; i < p->ref_cols.size(); ++i) {
    int c = p->ref_cols[i];
    std::snprintf(line, sizeof line, "ref %zu %s %s\n", i, t->names[c].c_str(), dtype_name(t->dtypes[c]));
    s += line;
  }
  for (size_t i = 0; i < p->proj_cols.size(); ++i) {
    int c = p->proj_cols[i];
    std::snprintf(line, sizeof line, "proj %zu %s %s %d\n", i, t->names[c].c_str(), dtype_name(t->dtypes[c]),
                  p->proj_ref[i]);
    s += line;
  }
  for (int pc = 0; pc < p->ninstr; ++pc) {
    const Instr &I = p->code[pc];
    switch (I.op) {
      case OP_RANGE:
        std::snprintf(line, sizeof line, "instr %d RANGE %d %s %" PRId64 " %" PRId64 "\n", pc, I.ref,
                      dtype_name(I.dtype), I.lo, I.hi);
        break;
      case OP_IN: {
        std::snprintf(line, sizeof line, "instr %d IN %d %s", pc, I.ref, dtype_name(I.dtype));
        s += line;
        for (int k = 0; k < I.n; ++k) {
          std::snprintf(line, sizeof line, "%s%" PRId64, k ? "," : " ", p->pool[I.off + k]);
          s += line;
        }
        line[0] = '\n';
        line[1] = 0;
        break;
      }
      case OP_UDF:
        std::snprintf(line, sizeof line, "instr %d UDF %d %s %d %s %" PRId64 " %" PRId64 " %" PRId64 "\n", pc, I.ref,
                      dtype_name(I.dtype), I.ref2, dtype_name(I.dtype2), p->pool[I.off], I.lo, I.hi);
        break;
      case OP_INSET: {
        std::snprintf(line, sizeof line, "instr %d IN %d %s", pc, I.ref, dtype_name(I.dtype));
        s += line;
        for (int k = 0; k < I.n; ++k) {
          std::snprintf(line, sizeof line, "%s%" PRId64, k ? "," : " ", p->pool[I.lo + k]);
          s += line;
        }
        line[0] = '\n';
        line[1] = 0;
        break;
      }
      case OP_JZ: std::snprintf(line, sizeof line, "instr %d JZ %d\n", pc, I.off); break;
      case OP_JNZ: std::snprintf(line, sizeof line, "instr %d JNZ %d\n", pc, I.off); break;
      case OP_AND: std::snprintf(line, sizeof line, "instr %d AND\n", pc); break;
      case OP_OR: std::snprintf(line, sizeof line, "instr %d OR\n", pc); break;
      case OP_NOT: std::snprintf(line, sizeof line, "instr %d NOT\n", pc); break;
      case OP_TRUE: std::snprintf(line, sizeof line, "instr %d TRUE\n", pc); break;
      case OP_FALSE: std::snprintf(line, sizeof line, "instr %d FALSE\n", pc); break;
    }
    s += line;
  }
  if (s.size() + 1 > buflen) return fail(ESC_EINVAL, "esc_predicate_explain: buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return ESC_OK;
}

}  // extern "C"
