"""Oracle interpreter for textual stencil programs (test infrastructure only).

The textual form restates the paper's stencil dialect (§IV): ``input`` names
the loaded fields (stencil.load), ``stage`` defines one stencil.apply whose body
reads earlier values at constant offsets (stencil.access) and returns one or
more results (stencil.return), ``column`` solves a tridiagonal system along k
per (i, j) column (the Thomas algorithm of §VII-B), and ``output`` names the
values stored over the domain (stencil.store).

    input in, coeff
    param dtr
    stage lap = 4.0*in - in[-1,0,0] - in[1,0,0] - in[0,-1,0] - in[0,1,0]
    stage flx = { let f = lap[1,0,0] - lap; return select(f*(in[1,0,0]-in) > 0, 0.0, f) }
    column x = thomas(a, b, c, d)
    output out

Expressions: numbers, names (offset [0,0,0]), name[di,dj,dk], unary -, + - * /
(left-associative, * and / bind tighter), min(a,b), max(a,b), abs(a),
select(x OP y, a, b) with OP in > < >= <=, and two level intrinsics: ``kpos``
(k minus the domain's lower k bound) and ``ksize`` (domain extent in k).
Control flow inside an operator (§IV-C, scf.if with scf.yield) is written

    if (x OP y) { let t = ...; yield a } else { yield b }

an expression whose value is the yield of the region the condition picks;
each region may bind its own lets. At a point only that region is evaluated.

Shape inference follows §V-B: statements are walked in reverse; a value's
range is the bounding box of the extents its consumers read (an output's
range is the domain; a stage consumer reads its own range shifted by each
access offset; a column consumer reads its i/j range over the whole domain
column). The staged interpreter evaluates each statement over its range; the
inlined interpreter evaluates one point at a time, recomputing producers at the
offsets read (§V-A), memoised per (value, point), which changes no bits.

This module is written independently of the CUDA library's parser.
"""

from __future__ import annotations

import re
from dataclasses import dataclass, field

import numpy as np

from .stencils import Grid, thomas

# ----------------------------------------------------------------------------
# parsing
# ----------------------------------------------------------------------------

_TOKEN = re.compile(r"\s*(?:(#[^\n]*)|(\d+\.\d*(?:[eE][-+]?\d+)?|\.\d+(?:[eE][-+]?\d+)?|\d+(?:[eE][-+]?\d+)?)"
                    r"|([A-Za-z_]\w*)|(>=|<=|[-+*/(),\[\]{}=;<>]))")


class ParseError(ValueError):
    pass


def _tokens(src: str):
    pos, out = 0, []
    while pos < len(src):
        m = _TOKEN.match(src, pos)
        if not m:
            if src[pos:].strip() == "":
                break
            raise ParseError(f"bad character at {pos}: {src[pos:pos + 10]!r}")
        pos = m.end()
        if m.group(1):
            continue
        if m.group(2):
            out.append(("num", m.group(2)))
        elif m.group(3):
            out.append(("id", m.group(3)))
        elif m.group(4):
            out.append(("op", m.group(4)))
    out.append(("eof", ""))
    return out


# expression nodes are tuples:
#   ("num", value) ("acc", name, (di,dj,dk)) ("ref", name) ("param", name) ("kpos",) ("ksize",)
#   ("neg", e) ("bin", op, a, b) ("min", a, b) ("max", a, b) ("abs", a) ("sel", rel, x, y, a, b)
#   ("if", rel, x, y, then_lets, then_yield, else_lets, else_yield), lets as [(name, expr)]


@dataclass
class Stmt:
    kind: str                      # "stage" | "column"
    results: list
    lets: list = field(default_factory=list)     # [(name, expr)]
    rets: list = field(default_factory=list)     # [expr] (stage)
    args: list = field(default_factory=list)     # [name] (column: a, b, c, d...)


@dataclass
class Program:
    inputs: list
    params: list
    stmts: list
    outputs: list


class _Parser:
    def __init__(self, src):
        self.t = _tokens(src)
        self.i = 0

    def peek(self, k=0):
        return self.t[self.i + k]

    def next(self):
        tok = self.t[self.i]
        self.i += 1
        return tok

    def expect(self, kind, val=None):
        tok = self.next()
        if tok[0] != kind or (val is not None and tok[1] != val):
            raise ParseError(f"expected {val or kind}, got {tok[1]!r}")
        return tok[1]

    def accept(self, val):
        if self.peek()[0] == "op" and self.peek()[1] == val:
            self.i += 1
            return True
        return False

    def names(self):
        out = [self.expect("id")]
        while self.accept(","):
            out.append(self.expect("id"))
        return out

    def integer(self):
        neg = self.accept("-")
        if not neg:
            self.accept("+")
        v = self.expect("num")
        if not re.fullmatch(r"\d+", v):
            raise ParseError(f"offset must be an integer: {v}")
        return -int(v) if neg else int(v)

    def primary(self, scope):
        kind, val = self.next()
        if kind == "num":
            return ("num", float(val))
        if kind == "op" and val == "(":
            e = self.expr(scope)
            self.expect("op", ")")
            return e
        if kind != "id":
            raise ParseError(f"unexpected {val!r}")
        if val in ("min", "max"):
            self.expect("op", "(")
            a = self.expr(scope)
            self.expect("op", ",")
            b = self.expr(scope)
            self.expect("op", ")")
            return (val, a, b)
        if val == "abs":
            self.expect("op", "(")
            a = self.expr(scope)
            self.expect("op", ")")
            return ("abs", a)
        if val == "select":
            self.expect("op", "(")
            x = self.expr(scope)
            rel = self.next()
            if rel[0] != "op" or rel[1] not in (">", "<", ">=", "<="):
                raise ParseError("select needs a comparison")
            y = self.expr(scope)
            self.expect("op", ",")
            a = self.expr(scope)
            self.expect("op", ",")
            b = self.expr(scope)
            self.expect("op", ")")
            return ("sel", rel[1], x, y, a, b)
        if val == "if":
            self.expect("op", "(")
            x = self.expr(scope)
            rel = self.next()
            if rel[0] != "op" or rel[1] not in (">", "<", ">=", "<="):
                raise ParseError("if needs a comparison")
            y = self.expr(scope)
            self.expect("op", ")")
            tl, te = self.region(scope)
            self.expect("id", "else")
            fl, fe = self.region(scope)
            return ("if", rel[1], x, y, tl, te, fl, fe)
        if val == "kpos":
            return ("kpos",)
        if val == "ksize":
            return ("ksize",)
        if self.accept("["):
            di = self.integer()
            self.expect("op", ",")
            dj = self.integer()
            self.expect("op", ",")
            dk = self.integer()
            self.expect("op", "]")
            if scope.get(val) not in ("field", "value"):
                raise ParseError(f"offset access to {val!r}, which is not a field or stage result")
            return ("acc", val, (di, dj, dk))
        cls = scope.get(val)
        if cls in ("field", "value"):
            return ("acc", val, (0, 0, 0))
        if cls == "let":
            return ("ref", val)
        if cls == "param":
            return ("param", val)
        raise ParseError(f"unknown name {val!r}")

    def region(self, scope):
        """{ let n = e; ... yield e }: the region's lets (visible in it only)
        and its yielded value."""
        self.expect("op", "{")
        local, lets = dict(scope), []
        while self.peek() == ("id", "let"):
            self.next()
            n = self.expect("id")
            self.expect("op", "=")
            e = self.expr(local)
            if n in local or n in _RESERVED:
                raise ParseError(f"let {n!r} shadows a name")
            local[n] = "let"
            lets.append((n, e))
            self.accept(";")
        self.expect("id", "yield")
        e = self.expr(local)
        self.accept(";")
        self.expect("op", "}")
        return lets, e

    def unary(self, scope):
        if self.accept("-"):
            return ("neg", self.unary(scope))
        return self.primary(scope)

    def term(self, scope):
        e = self.unary(scope)
        while self.peek() in (("op", "*"), ("op", "/")):
            op = self.next()[1]
            e = ("bin", op, e, self.unary(scope))
        return e

    def expr(self, scope):
        e = self.term(scope)
        while self.peek() in (("op", "+"), ("op", "-")):
            op = self.next()[1]
            e = ("bin", op, e, self.term(scope))
        return e

    def program(self) -> Program:
        inputs, params, stmts, outputs = [], [], [], []
        scope = {}

        def define(name, cls):
            if name in scope or name in _RESERVED:
                raise ParseError(f"name {name!r} defined twice or reserved")
            scope[name] = cls

        while self.peek()[0] != "eof":
            kw = self.expect("id")
            if kw == "input":
                for n in self.names():
                    define(n, "field")
                    inputs.append(n)
            elif kw == "param":
                for n in self.names():
                    define(n, "param")
                    params.append(n)
            elif kw == "output":
                for n in self.names():
                    if scope.get(n) != "value":
                        raise ParseError(f"output {n!r} is not a stage result")
                    outputs.append(n)
            elif kw == "stage":
                res = self.names()
                self.expect("op", "=")
                st = Stmt("stage", res)
                local = dict(scope)
                if self.accept("{"):
                    while self.peek() == ("id", "let"):
                        self.next()
                        n = self.expect("id")
                        self.expect("op", "=")
                        e = self.expr(local)
                        if n in local or n in _RESERVED:
                            raise ParseError(f"let {n!r} shadows a name")
                        local[n] = "let"
                        st.lets.append((n, e))
                        self.accept(";")
                    self.expect("id", "return")
                    st.rets.append(self.expr(local))
                    while self.accept(","):
                        st.rets.append(self.expr(local))
                    self.accept(";")
                    self.expect("op", "}")
                else:
                    st.rets.append(self.expr(local))
                if len(st.rets) != len(res):
                    raise ParseError("number of results and returned values differ")
                for n in res:
                    define(n, "value")
                stmts.append(st)
            elif kw == "column":
                res = self.names()
                self.expect("op", "=")
                self.expect("id", "thomas")
                self.expect("op", "(")
                args = self.names()
                self.expect("op", ")")
                if len(args) < 4 or len(res) != len(args) - 3:
                    raise ParseError("thomas(a, b, c, d1, ..., dn) yields n results")
                for a in args:
                    if scope.get(a) != "value":
                        raise ParseError(f"thomas argument {a!r} is not a stage result")
                for n in res:
                    define(n, "value")
                stmts.append(Stmt("column", res, args=args))
            else:
                raise ParseError(f"unknown statement {kw!r}")
        if not outputs:
            raise ParseError("program stores no output")
        return Program(inputs, params, stmts, outputs)


_RESERVED = ("min", "max", "abs", "select", "kpos", "ksize", "let", "return", "if", "else", "yield")


def parse(src: str) -> Program:
    return _Parser(src).program()


# ----------------------------------------------------------------------------
# shape inference (§V-B)
# ----------------------------------------------------------------------------

def _accesses(e, out):
    tag = e[0]
    if tag == "acc":
        out.append((e[1], e[2]))
    elif tag in ("neg", "abs"):
        _accesses(e[1], out)
    elif tag == "bin":
        _accesses(e[2], out)
        _accesses(e[3], out)
    elif tag in ("min", "max"):
        _accesses(e[1], out)
        _accesses(e[2], out)
    elif tag == "sel":
        for s in e[2:]:
            _accesses(s, out)
    elif tag == "if":   # both regions' accesses: either may run at a point of the range
        _accesses(e[2], out)
        _accesses(e[3], out)
        for lets, y in ((e[4], e[5]), (e[6], e[7])):
            for _, x in lets:
                _accesses(x, out)
            _accesses(y, out)
    return out


def _grow(rng, box):
    if rng is None:
        return [list(b) for b in box]
    return [[min(r[0], b[0]), max(r[1], b[1])] for r, b in zip(rng, box)]


def infer_ranges(prog: Program, lb, ub):
    """Range ([i0,i1],[j0,j1],[k0,k1]) of every input and statement result."""
    dom = [[lb[d], ub[d]] for d in range(3)]
    rng = {}
    for n in prog.outputs:
        rng[n] = _grow(rng.get(n), dom)
    for st in reversed(prog.stmts):
        box = None
        for n in st.results:
            if rng.get(n) is not None:
                box = _grow(box, rng[n])
        if box is None:
            continue                       # dead statement: no consumer
        for n in st.results:               # every result of one apply shares its domain
            rng[n] = box
        if st.kind == "stage":
            acc = []
            for _, e in st.lets:
                _accesses(e, acc)
            for e in st.rets:
                _accesses(e, acc)
            for name, (di, dj, dk) in acc:
                shifted = [[box[0][0] + di, box[0][1] + di], [box[1][0] + dj, box[1][1] + dj],
                           [box[2][0] + dk, box[2][1] + dk]]
                rng[name] = _grow(rng.get(name), shifted)
        else:
            if box[2] != dom[2]:
                raise ValueError("a column solve result is read outside the domain's k range")
            for name in st.args:
                rng[name] = _grow(rng.get(name), box)
    return {k: tuple(tuple(v) for v in r) for k, r in rng.items()}


def input_halo(prog: Program, lb, ub):
    """Per input: (lower, upper) extension of its inferred range beyond the domain."""
    r = infer_ranges(prog, lb, ub)
    out = {}
    for n in prog.inputs:
        if n not in r:
            out[n] = None
            continue
        out[n] = tuple((lb[d] - r[n][d][0], r[n][d][1] - ub[d]) for d in range(3))
    return out


# ----------------------------------------------------------------------------
# staged interpreter
# ----------------------------------------------------------------------------

_REL = {">": np.greater, "<": np.less, ">=": np.greater_equal, "<=": np.less_equal}


def _eval_box(e, box, env, lets, params, kdom):
    tag = e[0]
    if tag == "num":
        return np.float64(e[1])
    if tag == "acc":
        di, dj, dk = e[2]
        return env[e[1]].at(box, di, dj, dk)
    if tag == "ref":
        return lets[e[1]]
    if tag == "param":
        return np.float64(params[e[1]])
    if tag == "kpos":
        (_, _), (_, _), (k0, k1) = box
        return (np.arange(k0, k1, dtype=np.float64) - kdom[0]).reshape(-1, 1, 1)
    if tag == "ksize":
        return np.float64(kdom[1] - kdom[0])
    ev = lambda x: _eval_box(x, box, env, lets, params, kdom)
    if tag == "neg":
        return -ev(e[1])
    if tag == "bin":
        a, b = ev(e[2]), ev(e[3])
        return {"+": np.add, "-": np.subtract, "*": np.multiply, "/": np.divide}[e[1]](a, b)
    if tag == "min":
        return np.minimum(ev(e[1]), ev(e[2]))
    if tag == "max":
        return np.maximum(ev(e[1]), ev(e[2]))
    if tag == "abs":
        return np.abs(ev(e[1]))
    if tag == "sel":
        return np.where(_REL[e[1]](ev(e[2]), ev(e[3])), ev(e[4]), ev(e[5]))
    if tag == "if":
        # over a box each region is evaluated everywhere and the condition
        # picks per point; regions are pure, so every point gets the value of
        # the region that runs there
        def region(rlets, y):
            loc = dict(lets)
            for n, x in rlets:
                loc[n] = _eval_box(x, box, env, loc, params, kdom)
            return _eval_box(y, box, env, loc, params, kdom)
        return np.where(_REL[e[1]](ev(e[2]), ev(e[3])), region(e[4], e[5]), region(e[6], e[7]))
    raise ValueError(tag)


def _shape_of(box):
    (i0, i1), (j0, j1), (k0, k1) = box
    return (k1 - k0, j1 - j0, i1 - i0)


def run_staged(src_or_prog, fields: dict, lb, ub, params=None):
    """Evaluate a program stage by stage; returns {output name: array over [lb, ub)}.

    ``fields`` maps input names to Grids (logical coordinates)."""
    prog = parse(src_or_prog) if isinstance(src_or_prog, str) else src_or_prog
    params = dict(params or {})
    rng = infer_ranges(prog, lb, ub)
    env = dict(fields)
    kdom = (lb[2], ub[2])
    with np.errstate(divide="ignore", invalid="ignore"):
        for st in prog.stmts:
            box = rng.get(st.results[0])
            if box is None:
                continue
            shape = _shape_of(box)
            lo = (box[0][0], box[1][0], box[2][0])
            if st.kind == "stage":
                lets = {}
                for n, e in st.lets:
                    lets[n] = np.broadcast_to(_eval_box(e, box, env, lets, params, kdom), shape)
                for n, e in zip(st.results, st.rets):
                    env[n] = Grid(np.broadcast_to(_eval_box(e, box, env, lets, params, kdom), shape).copy(), lo)
            else:
                a, b, c = (env[x].at(box) for x in st.args[:3])
                for n, dname in zip(st.results, st.args[3:]):
                    env[n] = Grid(thomas(a, b, c, env[dname].at(box)), lo)
    box = ((lb[0], ub[0]), (lb[1], ub[1]), (lb[2], ub[2]))
    return {n: env[n].at(box).copy() for n in prog.outputs}


# ----------------------------------------------------------------------------
# inlined (per point) interpreter
# ----------------------------------------------------------------------------

def run_inlined(src_or_prog, fields: dict, lb, ub, params=None, points=None):
    """Evaluate outputs one point at a time, recomputing producers at every
    offset they are read at (§V-A). ``points``: optional list of (i, j, k);
    default all points of [lb, ub). Returns {name: {point: value}}."""
    prog = parse(src_or_prog) if isinstance(src_or_prog, str) else src_or_prog
    params = dict(params or {})
    owner = {}
    for st in prog.stmts:
        for idx, n in enumerate(st.results):
            owner[n] = (st, idx)
    memo = {}
    kdom = (lb[2], ub[2])

    def value(name, i, j, k):
        if name in fields:
            return fields[name].value(i, j, k)
        key = (name, i, j, k)
        if key in memo:
            return memo[key]
        st, idx = owner[name]
        if st.kind == "stage":
            lets = {}
            for n, e in st.lets:
                lets[n] = ev(e, i, j, k, lets)
            for n, e in zip(st.results, st.rets):
                memo[(n, i, j, k)] = ev(e, i, j, k, lets)
        else:
            K = kdom[1] - kdom[0]
            col = lambda a: np.array([value(a, i, j, kk) for kk in range(kdom[0], kdom[1])]).reshape(K, 1, 1)
            a, b, c = (col(x) for x in st.args[:3])
            for n, dname in zip(st.results, st.args[3:]):
                x = thomas(a, b, c, col(dname)).reshape(-1)
                for kk in range(K):
                    memo[(n, i, j, kdom[0] + kk)] = float(x[kk])
        return memo[key]

    def ev(e, i, j, k, lets):
        tag = e[0]
        if tag == "num":
            return e[1]
        if tag == "acc":
            di, dj, dk = e[2]
            return value(e[1], i + di, j + dj, k + dk)
        if tag == "ref":
            return lets[e[1]]
        if tag == "param":
            return float(params[e[1]])
        if tag == "kpos":
            return float(k - kdom[0])
        if tag == "ksize":
            return float(kdom[1] - kdom[0])
        if tag == "neg":
            return -ev(e[1], i, j, k, lets)
        if tag == "bin":
            a, b = ev(e[2], i, j, k, lets), ev(e[3], i, j, k, lets)
            op = e[1]
            if op == "+":
                return a + b
            if op == "-":
                return a - b
            if op == "*":
                return a * b
            return float(np.float64(a) / np.float64(b)) if b == 0 else a / b
        if tag == "min":
            return float(np.minimum(ev(e[1], i, j, k, lets), ev(e[2], i, j, k, lets)))
        if tag == "max":
            return float(np.maximum(ev(e[1], i, j, k, lets), ev(e[2], i, j, k, lets)))
        if tag == "abs":
            return abs(ev(e[1], i, j, k, lets))
        if tag == "sel":
            x, y = ev(e[2], i, j, k, lets), ev(e[3], i, j, k, lets)
            cond = {">": x > y, "<": x < y, ">=": x >= y, "<=": x <= y}[e[1]]
            # both branches are evaluated, as select does on value-semantic temps
            a, b = ev(e[4], i, j, k, lets), ev(e[5], i, j, k, lets)
            return a if cond else b
        if tag == "if":   # only the region the condition picks runs (scf.if)
            x, y = ev(e[2], i, j, k, lets), ev(e[3], i, j, k, lets)
            cond = {">": x > y, "<": x < y, ">=": x >= y, "<=": x <= y}[e[1]]
            rlets, yv = (e[4], e[5]) if cond else (e[6], e[7])
            loc = dict(lets)
            for n, x in rlets:
                loc[n] = ev(x, i, j, k, loc)
            return ev(yv, i, j, k, loc)
        raise ValueError(tag)

    if points is None:
        points = [(i, j, k) for k in range(lb[2], ub[2]) for j in range(lb[1], ub[1]) for i in range(lb[0], ub[0])]
    with np.errstate(divide="ignore", invalid="ignore"):
        return {n: {p: value(n, *p) for p in points} for n in prog.outputs}
