// ir.h - in-memory form of a stencil program (paper §IV) and the host passes
// on it: parsing of the textual form, verification, canonical printing (used to
// recognise the programs that have hand-written kernels), and shape inference
// (paper §V-B).
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace oec {

enum class Op : uint8_t {
  Num, Acc, Let, Param, KPos, KSize,       // leaves
  Neg, Abs,                                // unary
  Add, Sub, Mul, Div, Min, Max,            // binary
  Sel                                      // select(x REL y, a, b)
};
enum class Rel : uint8_t { GT, LT, GE, LE };

struct Expr {
  Op op = Op::Num;
  Rel rel = Rel::GT;
  double num = 0.0;       // Num
  int ref = -1;           // Acc: value id; Let: let id; Param: param id
  int off[3] = {0, 0, 0}; // Acc: constant offset (stencil.access)
  int a = -1, b = -1, c = -1, d = -1;  // children (expression ids)
};

enum class ValueKind : uint8_t { Input, Stage, Column };

struct Value {
  std::string name;
  ValueKind kind = ValueKind::Input;
  int stmt = -1;          // defining statement (Stage/Column)
  int index = 0;          // which result of the statement; input position for Input
};

enum class StmtKind : uint8_t { Stage, Column };

struct Stmt {
  StmtKind kind = StmtKind::Stage;
  std::vector<int> results;             // value ids
  std::vector<std::pair<int, int>> lets;  // (let id, expr id), in order
  std::vector<int> rets;                // expr ids (Stage)
  std::vector<int> args;                // value ids a, b, c, d... (Column)
};

struct Program {
  std::vector<Expr> pool;
  std::vector<Value> values;
  std::vector<int> inputs;              // value ids, declaration order
  std::vector<std::string> params;
  std::vector<std::string> lets;
  std::vector<Stmt> stmts;
  std::vector<int> outputs;             // value ids
};

// Parse and verify. Returns true on success; on failure `err` holds a message
// with the line number.
bool parse(const char* src, Program& out, std::string& err);

// Name-independent printing of the program's structure and constants (exact
// hexadecimal numbers); two programs with the same canonical text compute the
// same thing with the same inputs, params and outputs in the same order.
std::string canonical(const Program& p);

struct Box {
  int64_t lo[3] = {0, 0, 0};
  int64_t hi[3] = {0, 0, 0};
  bool valid = false;      // false: nothing reads this value
  int64_t volume() const {
    if (!valid) return 0;
    int64_t v = 1;
    for (int d = 0; d < 3; ++d) v *= (hi[d] > lo[d] ? hi[d] - lo[d] : 0);
    return v;
  }
};

// Shape inference (paper §V-B): the range of every value for the domain
// [lb, ub), indexed by value id. Returns false (with `err`) when a column
// solve's results would be needed outside the domain's k range.
bool infer_ranges(const Program& p, const int64_t lb[3], const int64_t ub[3], std::vector<Box>& ranges,
                  std::string& err);

// All stencil.access offsets (value id, offset) of a statement.
void stmt_accesses(const Program& p, const Stmt& s, std::vector<std::pair<int, std::array<int, 3>>>& out);

}  // namespace oec
