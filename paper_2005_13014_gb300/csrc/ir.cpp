// ir.cpp - parser, verifier, canonical printer and shape inference for the
// textual stencil-program form (paper §IV; shape inference paper §V-B).
#include "ir.h"

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <stdexcept>

namespace oec {
namespace {

struct Tok {
  enum Kind { Num, Id, Sym, End } kind;
  std::string text;
  int line;
};

struct ParseFail : std::runtime_error {
  using std::runtime_error::runtime_error;
};

std::vector<Tok> lex(const char* s) {
  std::vector<Tok> out;
  int line = 1;
  size_t i = 0, n = std::strlen(s);
  while (i < n) {
    char c = s[i];
    if (c == '\n') { ++line; ++i; continue; }
    if (std::isspace((unsigned char)c)) { ++i; continue; }
    if (c == '#') { while (i < n && s[i] != '\n') ++i; continue; }
    if (std::isdigit((unsigned char)c) || (c == '.' && i + 1 < n && std::isdigit((unsigned char)s[i + 1]))) {
      size_t j = i;
      while (j < n && std::isdigit((unsigned char)s[j])) ++j;
      if (j < n && s[j] == '.') { ++j; while (j < n && std::isdigit((unsigned char)s[j])) ++j; }
      if (j < n && (s[j] == 'e' || s[j] == 'E')) {
        size_t k = j + 1;
        if (k < n && (s[k] == '+' || s[k] == '-')) ++k;
        if (k < n && std::isdigit((unsigned char)s[k])) {
          j = k;
          while (j < n && std::isdigit((unsigned char)s[j])) ++j;
        }
      }
      out.push_back({Tok::Num, std::string(s + i, j - i), line});
      i = j;
      continue;
    }
    if (std::isalpha((unsigned char)c) || c == '_') {
      size_t j = i;
      while (j < n && (std::isalnum((unsigned char)s[j]) || s[j] == '_')) ++j;
      out.push_back({Tok::Id, std::string(s + i, j - i), line});
      i = j;
      continue;
    }
    if ((c == '>' || c == '<') && i + 1 < n && s[i + 1] == '=') {
      out.push_back({Tok::Sym, std::string(s + i, 2), line});
      i += 2;
      continue;
    }
    if (std::strchr("+-*/(),[]{}=;<>", c)) {
      out.push_back({Tok::Sym, std::string(1, c), line});
      ++i;
      continue;
    }
    char buf[96];
    std::snprintf(buf, sizeof buf, "line %d: unexpected character '%c'", line, c);
    throw ParseFail(buf);
  }
  out.push_back({Tok::End, "", line});
  return out;
}

enum class NameKind { Field, Value, Param, Let };

struct Parser {
  std::vector<Tok> t;
  size_t pos = 0;
  Program& p;
  std::map<std::string, std::pair<NameKind, int>> scope;  // name -> (kind, id)
  Stmt* cur = nullptr;   // the stage being parsed (its lets receive the regions' lets)

  Parser(const char* src, Program& prog) : t(lex(src)), p(prog) {}

  [[noreturn]] void fail(const std::string& what) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "line %d: ", t[pos < t.size() ? pos : t.size() - 1].line);
    throw ParseFail(buf + what);
  }
  const Tok& peek() const { return t[pos]; }
  bool is_sym(const char* s) const { return peek().kind == Tok::Sym && peek().text == s; }
  bool is_id(const char* s) const { return peek().kind == Tok::Id && peek().text == s; }
  bool accept(const char* s) {
    if (is_sym(s)) { ++pos; return true; }
    return false;
  }
  void expect(const char* s) {
    if (!accept(s)) fail(std::string("expected '") + s + "', got '" + peek().text + "'");
  }
  std::string ident() {
    if (peek().kind != Tok::Id) fail("expected a name, got '" + peek().text + "'");
    return t[pos++].text;
  }
  std::vector<std::string> names() {
    std::vector<std::string> v{ident()};
    while (accept(",")) v.push_back(ident());
    return v;
  }
  int integer() {
    bool neg = false;
    if (accept("-")) neg = true; else accept("+");
    if (peek().kind != Tok::Num || peek().text.find_first_not_of("0123456789") != std::string::npos)
      fail("offset must be an integer");
    long v = std::strtol(t[pos++].text.c_str(), nullptr, 10);
    if (v > 64) fail("offset larger than 64");
    return neg ? -int(v) : int(v);
  }
  int node(const Expr& e) {
    p.pool.push_back(e);
    return int(p.pool.size()) - 1;
  }
  static bool reserved(const std::string& n) {
    static const char* r[] = {"input", "param", "stage", "column", "output", "let", "return", "min", "max",
                              "abs", "select", "kpos", "ksize", "thomas", "if", "else", "yield"};
    for (const char* x : r) if (n == x) return true;
    return false;
  }
  void define(const std::string& n, NameKind k, int id) {
    if (reserved(n)) fail("'" + n + "' is a reserved word");
    if (scope.count(n)) fail("'" + n + "' defined twice");
    scope[n] = {k, id};
  }

  int primary() {
    const Tok tok = peek();
    if (tok.kind == Tok::Num) {
      ++pos;
      Expr e;
      e.op = Op::Num;
      e.num = std::strtod(tok.text.c_str(), nullptr);
      return node(e);
    }
    if (accept("(")) {
      int e = expr();
      expect(")");
      return e;
    }
    if (tok.kind != Tok::Id) fail("unexpected '" + tok.text + "'");
    ++pos;
    const std::string& n = tok.text;
    Expr e;
    if (n == "min" || n == "max") {
      expect("(");
      e.op = n == "min" ? Op::Min : Op::Max;
      e.a = expr();
      expect(",");
      e.b = expr();
      expect(")");
      return node(e);
    }
    if (n == "abs") {
      expect("(");
      e.op = Op::Abs;
      e.a = expr();
      expect(")");
      return node(e);
    }
    if (n == "select") {
      expect("(");
      e.op = Op::Sel;
      e.a = expr();
      if (accept(">")) e.rel = Rel::GT;
      else if (accept("<")) e.rel = Rel::LT;
      else if (accept(">=")) e.rel = Rel::GE;
      else if (accept("<=")) e.rel = Rel::LE;
      else fail("select needs a comparison");
      e.b = expr();
      expect(",");
      e.c = expr();
      expect(",");
      e.d = expr();
      expect(")");
      return node(e);
    }
    if (n == "if") {
      // if (x REL y) { lets; yield a } else { lets; yield b }: the value of
      // the region the condition picks (paper §IV-C, scf.if / scf.yield).
      // Regions are pure, so this is select(x REL y, a, b) with the regions'
      // lets bound in the enclosing stage (visible only inside their region).
      expect("(");
      e.op = Op::Sel;
      e.a = expr();
      if (accept(">")) e.rel = Rel::GT;
      else if (accept("<")) e.rel = Rel::LT;
      else if (accept(">=")) e.rel = Rel::GE;
      else if (accept("<=")) e.rel = Rel::LE;
      else fail("if needs a comparison");
      e.b = expr();
      expect(")");
      e.c = region();
      if (!is_id("else")) fail("expected 'else'");
      ++pos;
      e.d = region();
      return node(e);
    }
    if (n == "kpos") { e.op = Op::KPos; return node(e); }
    if (n == "ksize") { e.op = Op::KSize; return node(e); }
    auto it = scope.find(n);
    if (it == scope.end()) fail("unknown name '" + n + "'");
    NameKind k = it->second.first;
    if (accept("[")) {
      if (k != NameKind::Field && k != NameKind::Value) fail("offset access to '" + n + "', not a field or stage result");
      e.op = Op::Acc;
      e.ref = it->second.second;
      e.off[0] = integer();
      expect(",");
      e.off[1] = integer();
      expect(",");
      e.off[2] = integer();
      expect("]");
      return node(e);
    }
    switch (k) {
      case NameKind::Field:
      case NameKind::Value: e.op = Op::Acc; break;
      case NameKind::Param: e.op = Op::Param; break;
      case NameKind::Let: e.op = Op::Let; break;
    }
    e.ref = it->second.second;
    return node(e);
  }
  // { let n = e; ... yield e } of an if: its lets join the current stage's
  // lets (evaluated before the expression that holds the if) under names
  // visible in this region only; returns the yielded expression
  int region() {
    if (!cur) fail("if outside a stage");
    expect("{");
    std::vector<std::string> local;
    while (is_id("let")) {
      ++pos;
      std::string n = ident();
      expect("=");
      int e = expr();
      p.lets.push_back(n);
      int lid = int(p.lets.size()) - 1;
      define(n, NameKind::Let, lid);
      local.push_back(n);
      cur->lets.push_back({lid, e});
      accept(";");
    }
    if (!is_id("yield")) fail("expected 'yield'");
    ++pos;
    int v = expr();
    accept(";");
    expect("}");
    for (auto& n : local) scope.erase(n);
    return v;
  }
  int unary() {
    if (accept("-")) {
      Expr e;
      e.op = Op::Neg;
      e.a = unary();
      return node(e);
    }
    return primary();
  }
  int term() {
    int l = unary();
    while (is_sym("*") || is_sym("/")) {
      Expr e;
      e.op = t[pos++].text == "*" ? Op::Mul : Op::Div;
      e.a = l;
      e.b = unary();
      l = node(e);
    }
    return l;
  }
  int expr() {
    int l = term();
    while (is_sym("+") || is_sym("-")) {
      Expr e;
      e.op = t[pos++].text == "+" ? Op::Add : Op::Sub;
      e.a = l;
      e.b = term();
      l = node(e);
    }
    return l;
  }

  int new_value(const std::string& n, ValueKind k, int stmt, int index) {
    Value v;
    v.name = n;
    v.kind = k;
    v.stmt = stmt;
    v.index = index;
    p.values.push_back(v);
    int id = int(p.values.size()) - 1;
    define(n, k == ValueKind::Input ? NameKind::Field : NameKind::Value, id);
    return id;
  }

  void program() {
    while (peek().kind != Tok::End) {
      std::string kw = ident();
      if (kw == "input") {
        for (auto& n : names()) p.inputs.push_back(new_value(n, ValueKind::Input, -1, int(p.inputs.size())));
      } else if (kw == "param") {
        for (auto& n : names()) {
          p.params.push_back(n);
          define(n, NameKind::Param, int(p.params.size()) - 1);
        }
      } else if (kw == "output") {
        for (auto& n : names()) {
          auto it = scope.find(n);
          if (it == scope.end() || it->second.first != NameKind::Value) fail("output '" + n + "' is not a stage result");
          p.outputs.push_back(it->second.second);
        }
      } else if (kw == "stage") {
        std::vector<std::string> res = names();
        expect("=");
        Stmt st;
        st.kind = StmtKind::Stage;
        cur = &st;
        std::vector<std::string> local;
        if (accept("{")) {
          while (is_id("let")) {
            ++pos;
            std::string n = ident();
            expect("=");
            int e = expr();
            p.lets.push_back(n);
            int lid = int(p.lets.size()) - 1;
            define(n, NameKind::Let, lid);
            local.push_back(n);
            st.lets.push_back({lid, e});
            accept(";");
          }
          if (!is_id("return")) fail("expected 'return'");
          ++pos;
          st.rets.push_back(expr());
          while (accept(",")) st.rets.push_back(expr());
          accept(";");
          expect("}");
        } else {
          st.rets.push_back(expr());
        }
        cur = nullptr;
        for (auto& n : local) scope.erase(n);   // lets are local to their stage
        if (st.rets.size() != res.size()) fail("number of results and returned values differ");
        int sid = int(p.stmts.size());
        for (size_t r = 0; r < res.size(); ++r) st.results.push_back(new_value(res[r], ValueKind::Stage, sid, int(r)));
        p.stmts.push_back(st);
      } else if (kw == "column") {
        std::vector<std::string> res = names();
        expect("=");
        if (ident() != "thomas") fail("only thomas(...) column solves are supported");
        expect("(");
        std::vector<std::string> args = names();
        expect(")");
        if (args.size() < 4 || res.size() != args.size() - 3) fail("thomas(a, b, c, d1..dn) yields n results");
        Stmt st;
        st.kind = StmtKind::Column;
        for (auto& a : args) {
          auto it = scope.find(a);
          if (it == scope.end() || it->second.first != NameKind::Value) fail("thomas argument '" + a + "' is not a stage result");
          st.args.push_back(it->second.second);
        }
        int sid = int(p.stmts.size());
        for (size_t r = 0; r < res.size(); ++r) st.results.push_back(new_value(res[r], ValueKind::Column, sid, int(r)));
        p.stmts.push_back(st);
      } else {
        fail("unknown statement '" + kw + "'");
      }
    }
    if (p.outputs.empty()) fail("program stores no output");
  }
};

void print_expr(const Program& p, int id, std::string& s) {
  const Expr& e = p.pool[id];
  char buf[96];
  switch (e.op) {
    case Op::Num: std::snprintf(buf, sizeof buf, "%a", e.num); s += buf; return;
    case Op::Acc: {
      const Value& v = p.values[e.ref];
      if (v.kind == ValueKind::Input) std::snprintf(buf, sizeof buf, "I%d", v.index);
      else std::snprintf(buf, sizeof buf, "S%d.%d", v.stmt, v.index);
      s += buf;
      std::snprintf(buf, sizeof buf, "[%d,%d,%d]", e.off[0], e.off[1], e.off[2]);
      s += buf;
      return;
    }
    case Op::Let: std::snprintf(buf, sizeof buf, "L%d", e.ref); s += buf; return;
    case Op::Param: std::snprintf(buf, sizeof buf, "P%d", e.ref); s += buf; return;
    case Op::KPos: s += "kpos"; return;
    case Op::KSize: s += "ksize"; return;
    default: break;
  }
  static const char* names[] = {"", "", "", "", "", "", "neg", "abs", "add", "sub", "mul", "div", "min", "max", "sel"};
  s += names[int(e.op)];
  s += "(";
  if (e.op == Op::Sel) {
    static const char* rel[] = {">", "<", ">=", "<="};
    s += rel[int(e.rel)];
    s += ",";
  }
  int kids[4] = {e.a, e.b, e.c, e.d};
  bool first = true;
  for (int k : kids) {
    if (k < 0) continue;
    if (!first) s += ",";
    first = false;
    print_expr(p, k, s);
  }
  s += ")";
}

void collect_acc(const Program& p, int id, std::vector<std::pair<int, std::array<int, 3>>>& out) {
  const Expr& e = p.pool[id];
  if (e.op == Op::Acc) {
    out.push_back({e.ref, {e.off[0], e.off[1], e.off[2]}});
    return;
  }
  for (int k : {e.a, e.b, e.c, e.d})
    if (k >= 0) collect_acc(p, k, out);
}

// Local let ids are renumbered per statement for canonical printing.
void renumber_lets(const Program& src, Program& dst) {
  dst = src;
  for (auto& st : dst.stmts) {
    int next = 0;
    std::map<int, int> m;
    for (auto& l : st.lets) m[l.first] = next++;
    for (auto& l : st.lets) l.first = m[l.first];
    // rewrite Let refs inside this statement's expressions
    std::vector<int> stack;
    for (auto& l : st.lets) stack.push_back(l.second);
    for (int r : st.rets) stack.push_back(r);
    while (!stack.empty()) {
      int id = stack.back();
      stack.pop_back();
      Expr& e = dst.pool[id];
      if (e.op == Op::Let && m.count(e.ref)) e.ref = m[e.ref];
      for (int k : {e.a, e.b, e.c, e.d})
        if (k >= 0) stack.push_back(k);
    }
  }
}

}  // namespace

bool parse(const char* src, Program& out, std::string& err) {
  out = Program();
  try {
    if (!src) throw ParseFail("null source");
    Parser ps(src, out);
    ps.program();
    return true;
  } catch (const ParseFail& f) {
    err = f.what();
    return false;
  } catch (const std::exception& f) {
    err = std::string("parse error: ") + f.what();
    return false;
  }
}

std::string canonical(const Program& p0) {
  Program p;
  renumber_lets(p0, p);
  std::string s;
  char buf[64];
  std::snprintf(buf, sizeof buf, "in %zu param %zu\n", p.inputs.size(), p.params.size());
  s += buf;
  for (size_t i = 0; i < p.stmts.size(); ++i) {
    const Stmt& st = p.stmts[i];
    if (st.kind == StmtKind::Column) {
      s += "column(";
      for (int a : st.args) {
        const Value& v = p.values[a];
        std::snprintf(buf, sizeof buf, "S%d.%d,", v.stmt, v.index);
        s += buf;
      }
      s += ")\n";
      continue;
    }
    s += "stage{";
    for (auto& l : st.lets) {
      std::snprintf(buf, sizeof buf, "L%d=", l.first);
      s += buf;
      print_expr(p, l.second, s);
      s += ";";
    }
    s += "ret ";
    for (int r : st.rets) {
      print_expr(p, r, s);
      s += ";";
    }
    s += "}\n";
  }
  s += "out";
  for (int o : p.outputs) {
    const Value& v = p.values[o];
    std::snprintf(buf, sizeof buf, " S%d.%d", v.stmt, v.index);
    s += buf;
  }
  return s;
}

void stmt_accesses(const Program& p, const Stmt& s, std::vector<std::pair<int, std::array<int, 3>>>& out) {
  for (auto& l : s.lets) collect_acc(p, l.second, out);
  for (int r : s.rets) collect_acc(p, r, out);
}

static void grow(Box& b, const int64_t lo[3], const int64_t hi[3]) {
  if (!b.valid) {
    for (int d = 0; d < 3; ++d) { b.lo[d] = lo[d]; b.hi[d] = hi[d]; }
    b.valid = true;
    return;
  }
  for (int d = 0; d < 3; ++d) {
    if (lo[d] < b.lo[d]) b.lo[d] = lo[d];
    if (hi[d] > b.hi[d]) b.hi[d] = hi[d];
  }
}

bool infer_ranges(const Program& p, const int64_t lb[3], const int64_t ub[3], std::vector<Box>& r, std::string& err) {
  r.assign(p.values.size(), Box());
  for (int o : p.outputs) grow(r[o], lb, ub);
  std::vector<std::pair<int, std::array<int, 3>>> acc;
  for (int si = int(p.stmts.size()) - 1; si >= 0; --si) {
    const Stmt& st = p.stmts[si];
    Box box;
    for (int v : st.results)
      if (r[v].valid) grow(box, r[v].lo, r[v].hi);
    if (!box.valid) continue;                 // dead statement
    for (int v : st.results) r[v] = box;      // one iteration domain per apply
    if (st.kind == StmtKind::Stage) {
      acc.clear();
      stmt_accesses(p, st, acc);
      for (auto& a : acc) {
        int64_t lo[3], hi[3];
        for (int d = 0; d < 3; ++d) { lo[d] = box.lo[d] + a.second[d]; hi[d] = box.hi[d] + a.second[d]; }
        grow(r[a.first], lo, hi);
      }
    } else {
      if (box.lo[2] != lb[2] || box.hi[2] != ub[2]) {
        err = "a column solve result is read outside the domain's k range";
        return false;
      }
      for (int a : st.args) grow(r[a], box.lo, box.hi);
    }
  }
  return true;
}

}  // namespace oec
