"""A Python front end for the textual stencil-program form.

A stencil program is written as a Python function over symbolic fields; the
function is traced once (operator overloading, no execution on data) and the
trace is printed in the textual form that ``oec_program_create`` parses
(paper §IV: ``input`` loads, one ``stage`` per stencil.apply with constant
offset accesses, ``column`` solves, ``output`` stores). It plays the role of
the Python front ends that lower to the stencil dialect (GT4Py-like, paper
§VII-E). Nothing here computes: the library does, from the text.

    from paper_2005_13014_gb300 import dsl

    @dsl.program
    def hdiff(inp: dsl.Field, coeff: dsl.Field):
        lap = dsl.stage(4.0 * inp - inp[-1, 0, 0] - inp[1, 0, 0] - inp[0, -1, 0] - inp[0, 1, 0])
        ...
        return {"out": inp - coeff * (...)}

    hdiff.text          # the program text
    hdiff.compile("f64")  # an api.Program

Rules: offsets apply to named values (inputs, stages); indexing any other
expression makes it a stage first. ``let`` binds a subexpression locally in
the next stage (the text's ``let``). A program written with the same stages,
lets and operation order as one of the library's hand-written programs is
recognised as that program and runs its kernels. ``if_(a > b, x, y)`` is the
text's region ``if`` (the value of x where a > b holds, else of y).
``select(a > b, x, y)``, ``minimum``,
``maximum``, ``absolute``, ``kpos`` and ``ksize`` map to the text's
``select``, ``min``, ``max``, ``abs``, ``kpos`` and ``ksize``; ``thomas(a, b,
c, d...)`` is a column solve. Parameters are arguments annotated
``dsl.Param``.
"""

import inspect

__all__ = ["Field", "Param", "program", "stage", "let", "select", "if_", "minimum", "maximum", "absolute", "thomas",
           "kpos", "ksize", "Program"]


class Field:
    """Annotation of a program argument that is an input field."""


class Param:
    """Annotation of a program argument that is a scalar parameter."""


_ctx = []   # the trace being recorded (innermost last)


def _trace():
    if not _ctx:
        raise RuntimeError("stencil expressions are only valid inside a traced @dsl.program")
    return _ctx[-1]


def _num(v):
    r = repr(float(v))
    return r if ("e" in r or "." in r or "n" in r) else r + ".0"


def _wrap(v):
    if isinstance(v, Expr):
        return v
    if isinstance(v, (int, float)) and not isinstance(v, bool):
        return Expr(_num(v), prec=4 if v >= 0 else 3)
    raise TypeError(f"not a stencil expression: {v!r}")


class Expr:
    """A symbolic expression: its text and the precedence of its top
    operator (1 additive, 2 multiplicative, 3 unary, 4 atom)."""

    def __init__(self, text, prec=4):
        self.text, self.prec = text, prec

    def _par(self, p, right=False):
        # parenthesise when binding weaker, or equally on the right of a
        # left-associative operator (a - (b - c) keeps its grouping)
        return f"({self.text})" if self.prec < p or (right and self.prec == p) else self.text

    def _bin(self, op, other, p, swap=False):
        a, b = (_wrap(other), self) if swap else (self, _wrap(other))
        return Expr(f"{a._par(p)} {op} {b._par(p, right=True)}" if p == 1 else
                    f"{a._par(p)}{op}{b._par(p, right=True)}", p)

    def __add__(self, o): return self._bin("+", o, 1)
    def __radd__(self, o): return self._bin("+", o, 1, swap=True)
    def __sub__(self, o): return self._bin("-", o, 1)
    def __rsub__(self, o): return self._bin("-", o, 1, swap=True)
    def __mul__(self, o): return self._bin("*", o, 2)
    def __rmul__(self, o): return self._bin("*", o, 2, swap=True)
    def __truediv__(self, o): return self._bin("/", o, 2)
    def __rtruediv__(self, o): return self._bin("/", o, 2, swap=True)
    def __neg__(self): return Expr(f"-{self._par(3)}", 3)
    def __pos__(self): return self

    def _cmp(self, rel, o): return _Cond(self, rel, _wrap(o))
    def __gt__(self, o): return self._cmp(">", o)
    def __lt__(self, o): return self._cmp("<", o)
    def __ge__(self, o): return self._cmp(">=", o)
    def __le__(self, o): return self._cmp("<=", o)

    def __bool__(self):
        raise TypeError("stencil expressions have no truth value; use dsl.select")

    def __getitem__(self, off):
        return stage(self)[off]


class Value(Expr):
    """A named value (input or stage): indexable at constant offsets."""

    def __init__(self, name):
        super().__init__(name, 4)
        self.name = name

    def __getitem__(self, off):
        if not (isinstance(off, tuple) and len(off) == 3 and all(isinstance(x, int) for x in off)):
            raise TypeError("offsets are three integers [di, dj, dk]")
        if off == (0, 0, 0):
            return Expr(self.name)
        return Expr(f"{self.name}[{off[0]},{off[1]},{off[2]}]")


class _Cond:
    def __init__(self, a, rel, b):
        self.a, self.rel, self.b = a, rel, b

    def __bool__(self):
        raise TypeError("comparisons are only valid as the first argument of dsl.select")


class _Trace:
    def __init__(self):
        self.lines, self.names, self.n = [], set(), 0
        self.pending = []   # lets waiting for the next stage

    def fresh(self, hint="s"):
        while True:
            name = f"{hint}{self.n}"
            self.n += 1
            if name not in self.names:
                self.names.add(name)
                return name

    def claim(self, name):
        if name in self.names:
            raise ValueError(f"name {name!r} used twice")
        self.names.add(name)


def stage(expr, name=None):
    """One stencil.apply: name = expr, with the lets made since the previous
    stage as its local bindings. Returns the named value."""
    t = _trace()
    e = _wrap(expr)
    if name is None:
        name = t.fresh()
    else:
        t.claim(name)
    if t.pending:
        lets = "; ".join(f"let {n} = {x}" for n, x in t.pending)
        t.lines.append(f"stage {name} = {{ {lets}; return {e.text} }}")
        t.pending = []
    else:
        t.lines.append(f"stage {name} = {e.text}")
    return Value(name)


def let(expr, name=None):
    """A local binding of the next stage (the text's ``let``): evaluated once
    per point there, usable only in that stage's expression."""
    t = _trace()
    e = _wrap(expr)
    if name is None:
        name = t.fresh("l")
    else:
        t.claim(name)
    t.pending.append((name, e.text))
    return Expr(name)


def select(cond, a, b):
    if not isinstance(cond, _Cond):
        raise TypeError("select needs a comparison such as x > 0.0")
    a, b = _wrap(a), _wrap(b)
    return Expr(f"select({cond.a.text} {cond.rel} {cond.b.text}, {a.text}, {b.text})")


def if_(cond, then, otherwise):
    """Control flow inside a stage (paper §IV-C, scf.if): the value of
    ``then`` where the comparison holds, else of ``otherwise``; printed as the
    text's ``if (...) { yield ... } else { yield ... }``."""
    if not isinstance(cond, _Cond):
        raise TypeError("if_ needs a comparison such as x > 0.0")
    a, b = _wrap(then), _wrap(otherwise)
    return Expr(f"if ({cond.a.text} {cond.rel} {cond.b.text}) {{ yield {a.text} }} else {{ yield {b.text} }}")


def minimum(a, b):
    return Expr(f"min({_wrap(a).text}, {_wrap(b).text})")


def maximum(a, b):
    return Expr(f"max({_wrap(a).text}, {_wrap(b).text})")


def absolute(a):
    return Expr(f"abs({_wrap(a).text})")


kpos = Expr("kpos")
ksize = Expr("ksize")


def thomas(a, b, c, *rhs):
    """Column solve a x(k-1) + b x(k) + c x(k+1) = d for each right-hand side
    d (paper §VII-B's Thomas algorithm); returns the solutions."""
    if not rhs:
        raise ValueError("thomas needs at least one right-hand side")
    t = _trace()
    args = [v if isinstance(v, Value) else stage(v) for v in (a, b, c) + rhs]
    names = [t.fresh("x") for _ in rhs]
    t.lines.append(f"column {', '.join(names)} = thomas({', '.join(v.name for v in args)})")
    vals = [Value(n) for n in names]
    return vals[0] if len(vals) == 1 else tuple(vals)


class Program:
    """A traced program: ``text`` (the textual form), ``inputs``,
    ``params``, ``outputs``; ``compile(dtype)`` makes an ``api.Program``."""

    def __init__(self, fn):
        self.fn = fn
        self.__name__ = getattr(fn, "__name__", "program")
        sig = inspect.signature(fn)
        self.inputs, self.params = [], []
        for p in sig.parameters.values():
            (self.params if p.annotation is Param else self.inputs).append(p.name)
        t = _Trace()
        for n in self.inputs + self.params:
            t.claim(n)
        _ctx.append(t)
        try:
            res = fn(*[Value(n) for n in sig.parameters])
        finally:
            _ctx.pop()
        if isinstance(res, dict):
            items = list(res.items())
        else:
            items = [(None, r) for r in (res if isinstance(res, tuple) else (res,))]
        if t.pending:
            raise ValueError("dsl.let used by no stage (lets belong to the next stage)")
        self.outputs = []
        _ctx.append(t)
        try:
            for name, r in items:
                if isinstance(r, Value) and name in (None, r.name) and r.name not in self.inputs + self.params:
                    self.outputs.append(r.name)
                else:
                    self.outputs.append(stage(r, name).name)
        finally:
            _ctx.pop()
        head = [f"input {', '.join(self.inputs)}"]
        if self.params:
            head.append(f"param {', '.join(self.params)}")
        self.text = "\n".join(head + t.lines + [f"output {', '.join(self.outputs)}"]) + "\n"

    def compile(self, dtype="f64", generic=False):
        from .api import Program as _P
        return _P(self.text, dtype=dtype, generic=generic)

    def __repr__(self):
        return f"<dsl.Program {self.__name__}: {len(self.inputs)} inputs, {len(self.outputs)} outputs>"


def program(fn):
    """Decorator: trace ``fn`` into a ``Program``."""
    return Program(fn)
