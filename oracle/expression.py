"""Evaluator of expression integrands for the FP64 oracle.

TEST INFRASTRUCTURE (see zmc_oracle.py): only the tests, the smoke check and
the benchmark's CPU legs use it; it shares no code with the CUDA path, which
compiles the same text with NVRTC.

Sec. 3.3 and Sec. 4 of the paper ask for user integrands with condition
checks and special functions.  An expression integrand is one C expression in
the point's coordinates x[0..d-1] and the user's parameters p[0..]; this
module parses it with a recursive-descent parser that follows C's grammar
and operator precedence, and evaluates it in FP64 over an array of points:

  expr     := cond
  cond     := or ( '?' expr ':' cond )?            (right-associative)
  or       := and ( '||' and )*
  and      := equal ( '&&' equal )*
  equal    := rel ( ('==' | '!=') rel )*
  rel      := add ( ('<' | '<=' | '>' | '>=') add )*
  add      := mul ( ('+' | '-') mul )*
  mul      := unary ( ('*' | '/') unary )*
  unary    := ('-' | '+' | '!') unary | primary
  primary  := number | x '[' int ']' | p '[' int ']' | name '(' args ')'
              | '(' expr ')'

Comparisons and the logical operators give 1 or 0; a condition is true when
nonzero.  As in C, an integer literal is an int and int-by-int arithmetic
stays integer (1/2 is 0); anything that meets a coordinate, a parameter, a
function value or a floating literal is FP64.  Both branches of '?:' are
evaluated and the selected one is kept (floating-point evaluation has no side
effects to avoid).  Numbers may carry C's 'f' suffix.  Functions: the C math library's by their double and
float names (sin / sinf, ...) and the CUDA fast-math spellings (__sinf,
__expf, ...), all evaluated in FP64 here.
"""
from __future__ import annotations

import math
import re

import numpy as np

_TOKEN = re.compile(r"""
    \s*(?:
      (?P<num>(?:\d+\.\d*|\.\d+|\d+)(?:[eE][+-]?\d+)?[fFlL]?)
    | (?P<name>[A-Za-z_][A-Za-z_0-9]*)
    | (?P<op>\|\||&&|==|!=|<=|>=|[-+*/<>!?:()\[\],])
    )""", re.VERBOSE)


def _vec(f):
    v = np.vectorize(f, otypes=[np.float64])
    return lambda a: v(np.asarray(a, dtype=np.float64))


_UNARY = {
    "sin": np.sin, "cos": np.cos, "tan": np.tan, "asin": np.arcsin, "acos": np.arccos,
    "atan": np.arctan, "sinh": np.sinh, "cosh": np.cosh, "tanh": np.tanh,
    "exp": np.exp, "exp2": np.exp2, "expm1": np.expm1, "log": np.log, "log2": np.log2,
    "log10": np.log10, "log1p": np.log1p, "sqrt": np.sqrt, "cbrt": np.cbrt,
    "fabs": np.abs, "floor": np.floor, "ceil": np.ceil, "trunc": np.trunc,
    "erf": _vec(math.erf), "erfc": _vec(math.erfc), "lgamma": _vec(math.lgamma),
    "tgamma": _vec(math.gamma),
}
_BINARY = {"pow": np.power, "fmin": np.fmin, "fmax": np.fmax, "atan2": np.arctan2,
           "hypot": np.hypot, "fmod": np.fmod}
_TERNARY = {"fma": lambda a, b, c: a * b + c}


def _canonical(name: str) -> str:
    """C float and CUDA fast-math spellings -> the double function's name."""
    base = name[2:] if name.startswith("__") else name
    for table in (_UNARY, _BINARY, _TERNARY):
        if base in table:
            return base
        if base.endswith("f") and base[:-1] in table:
            return base[:-1]
    raise ValueError("unknown function in expression: %s" % name)


class Expression:
    """A parsed expression integrand; ``eval(x, p)`` for x of shape (N, d)."""

    def __init__(self, text: str):
        if text.startswith("expr:"):
            text = text[5:]
        self.text = text
        self._toks = self._tokenize(text)
        self._i = 0
        self._tree = self._cond()
        if self._i != len(self._toks):
            raise ValueError("unexpected %r in expression" % (self._toks[self._i][1],))

    # ------------------------------------------------------------ parsing
    @staticmethod
    def _tokenize(text):
        toks, pos = [], 0
        text = text.rstrip()
        while pos < len(text):
            m = _TOKEN.match(text, pos)
            if not m or m.end() == pos:
                raise ValueError("cannot read expression at %r" % text[pos:])
            kind = m.lastgroup
            toks.append((kind, m.group(kind)))
            pos = m.end()
        return toks

    def _peek(self):
        return self._toks[self._i][1] if self._i < len(self._toks) else None

    def _take(self, want=None):
        if self._i >= len(self._toks):
            raise ValueError("expression ends early")
        kind, val = self._toks[self._i]
        if want is not None and val != want:
            raise ValueError("expected %r, found %r" % (want, val))
        self._i += 1
        return kind, val

    def _cond(self):
        c = self._or()
        if self._peek() == "?":
            self._take("?")
            a = self._cond()
            self._take(":")
            b = self._cond()
            return ("?:", c, a, b)
        return c

    def _left(self, sub, ops):
        node = sub()
        while self._peek() in ops:
            op = self._take()[1]
            node = (op, node, sub())
        return node

    def _or(self):
        return self._left(self._and, ("||",))

    def _and(self):
        return self._left(self._equal, ("&&",))

    def _equal(self):
        return self._left(self._rel, ("==", "!="))

    def _rel(self):
        return self._left(self._add, ("<", "<=", ">", ">="))

    def _add(self):
        return self._left(self._mul, ("+", "-"))

    def _mul(self):
        return self._left(self._unary, ("*", "/"))

    def _unary(self):
        if self._peek() in ("-", "+", "!"):
            op = self._take()[1]
            return ("u" + op, self._unary())
        return self._primary()

    def _primary(self):
        kind, val = self._take()
        if kind == "num":
            # an integer literal is a C int (1/2 is 0); anything else a double
            return ("num", int(val) if val.isdigit() else float(val.rstrip("fFlL")))
        if val == "(":
            node = self._cond()
            self._take(")")
            return node
        if kind == "name" and val in ("x", "p") and self._peek() == "[":
            self._take("[")
            k, idx = self._take()
            if k != "num" or not idx.isdigit():
                raise ValueError("index of %s[] must be an integer literal" % val)
            self._take("]")
            return (val, int(idx))
        if kind == "name" and self._peek() == "(":
            self._take("(")
            args = [self._cond()]
            while self._peek() == ",":
                self._take(",")
                args.append(self._cond())
            self._take(")")
            return ("call", _canonical(val), args)
        raise ValueError("unexpected %r in expression" % val)

    # --------------------------------------------------------- evaluation
    def eval(self, x, p=()) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        p = np.asarray(p, dtype=np.float64)
        with np.errstate(all="ignore"):
            out = self._eval(self._tree, x, p)
        return np.broadcast_to(np.asarray(out, dtype=np.float64), x.shape[:1]).copy()

    def _eval(self, node, x, p):
        tag = node[0]
        if tag == "num":
            return node[1]
        if tag == "x":
            return x[:, node[1]]
        if tag == "p":
            return p[node[1]]
        if tag == "call":
            name, args = node[1], [self._eval(a, x, p) for a in node[2]]
            for table, arity in ((_UNARY, 1), (_BINARY, 2), (_TERNARY, 3)):
                if name in table:
                    if len(args) != arity:
                        raise ValueError("%s takes %d arguments" % (name, arity))
                    return table[name](*args)
        if tag == "?:":
            c = self._eval(node[1], x, p)
            return np.where(np.asarray(c) != 0, self._eval(node[2], x, p),
                            self._eval(node[3], x, p))
        if tag.startswith("u"):
            v = self._eval(node[1], x, p)
            if tag == "u-":
                return -v
            if tag == "u+":
                return v
            return int(v == 0) if isinstance(v, int) else np.where(np.asarray(v) == 0, 1.0, 0.0)
        a, b = self._eval(node[1], x, p), self._eval(node[2], x, p)
        if isinstance(a, int) and isinstance(b, int):
            return self._int_op(tag, a, b)
        if tag == "+":
            return a + b
        if tag == "-":
            return a - b
        if tag == "*":
            return a * b
        if tag == "/":
            return np.true_divide(a, b)
        if tag == "&&":
            return np.where((np.asarray(a) != 0) & (np.asarray(b) != 0), 1.0, 0.0)
        if tag == "||":
            return np.where((np.asarray(a) != 0) | (np.asarray(b) != 0), 1.0, 0.0)
        cmp = {"<": np.less, "<=": np.less_equal, ">": np.greater, ">=": np.greater_equal,
               "==": np.equal, "!=": np.not_equal}[tag]
        return np.where(cmp(a, b), 1.0, 0.0)

    @staticmethod
    def _int_op(tag, a, b):
        """C's int arithmetic: division truncates toward zero; comparisons and
        logic give 1 or 0."""
        if tag == "/":
            if b == 0:
                raise ValueError("integer division by zero in expression")
            q = abs(a) // abs(b)
            return q if (a >= 0) == (b >= 0) else -q
        ops = {"+": a + b, "-": a - b, "*": a * b, "<": a < b, "<=": a <= b, ">": a > b,
               ">=": a >= b, "==": a == b, "!=": a != b, "&&": bool(a) and bool(b),
               "||": bool(a) or bool(b)}
        return int(ops[tag])
