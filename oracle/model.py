"""Oracle: model expressions (test infrastructure only).

Section "Modeling Kernel Execution Time": a model is an output feature plus an
expression g over input features ``f_*`` and parameters ``p_*`` that is
differentiable in the parameters.  Section "Computing Model Parameters": the
Jacobian d g_k / d p_i is obtained by symbolic differentiation.  Section
"Modeling Operation Overlap" uses tanh; exp, log and sqrt are accepted too.

Grammar (recursive descent, in this order of precedence):
    expr  := term (('+' | '-') term)*
    term  := unary (('*' | '/') unary)*
    unary := '-' unary | prim
    prim  := NUMBER | NAME | FUNC '(' expr ')' | '(' expr ')'
A NAME starts with ``f_`` or ``p_`` and runs up to whitespace or one of
``+ * / ( )``; a ``-`` right after a name character belongs to the name (so a
binary minus after a name must be preceded by whitespace).
"""
import math
import re

FUNCS = ("tanh", "exp", "log", "sqrt")


def tokenize(s):
    toks, i = [], 0
    while i < len(s):
        ch = s[i]
        if ch.isspace():
            i += 1
        elif ch in "+-*/()":
            toks.append(ch)
            i += 1
        elif ch.isdigit() or (ch == "." and i + 1 < len(s) and s[i + 1].isdigit()):
            m = re.match(r"[0-9]*\.?[0-9]*(?:[eE][-+]?[0-9]+)?", s[i:])
            toks.append(("num", float(m.group(0))))
            i += len(m.group(0))
        elif ch.isalpha() or ch == "_":
            j = i
            while j < len(s) and not s[j].isspace() and s[j] not in "+*/()":
                j += 1
            toks.append(("name", s[i:j]))
            i = j
        else:
            raise ValueError("unexpected %r in model expression" % ch)
    return toks


class _P:
    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def take(self):
        tok = self.peek()
        self.i += 1
        return tok

    def expr(self):
        node = self.term()
        while self.peek() in ("+", "-"):
            op = self.take()
            node = (op, node, self.term())
        return node

    def term(self):
        node = self.unary()
        while self.peek() in ("*", "/"):
            op = self.take()
            node = (op, node, self.unary())
        return node

    def unary(self):
        if self.peek() == "-":
            self.take()
            return ("neg", self.unary())
        return self.prim()

    def prim(self):
        tok = self.take()
        if tok == "(":
            node = self.expr()
            if self.take() != ")":
                raise ValueError("missing ')'")
            return node
        if isinstance(tok, tuple) and tok[0] == "num":
            return ("num", tok[1])
        if isinstance(tok, tuple) and tok[0] == "name":
            name = tok[1]
            if name in FUNCS:
                if self.take() != "(":
                    raise ValueError("expected '(' after %s" % name)
                arg = self.expr()
                if self.take() != ")":
                    raise ValueError("missing ')'")
                return ("fn", name, arg)
            if name.startswith("f_"):
                return ("feat", name)
            if name.startswith("p_"):
                return ("par", name)
            raise ValueError("unknown name %r" % name)
        raise ValueError("unexpected token %r" % (tok,))


class Model:
    """Output feature + expression; parameters are ordered by first appearance."""

    def __init__(self, out_feature, expr):
        self.out_feature = out_feature
        self.expr = expr
        p = _P(tokenize(expr))
        self.tree = p.expr()
        if p.i != len(p.t):
            raise ValueError("trailing input in model expression")
        self.features, self.params = [], []

        def walk(n):
            if n[0] == "feat" and n[1] not in self.features:
                self.features.append(n[1])
            elif n[0] == "par" and n[1] not in self.params:
                self.params.append(n[1])
            for c in n[1:]:
                if isinstance(c, tuple):
                    walk(c)
        walk(self.tree)

    def eval(self, p, f):
        """g(p; f) for one row; p and f map names to floats."""
        def ev(n):
            k = n[0]
            if k == "num":
                return n[1]
            if k == "feat":
                return f[n[1]]
            if k == "par":
                return p[n[1]]
            if k == "neg":
                return -ev(n[1])
            if k == "fn":
                x = ev(n[2])
                return {"tanh": math.tanh, "exp": math.exp, "log": math.log, "sqrt": math.sqrt}[n[1]](x)
            a, b = ev(n[1]), ev(n[2])
            if k == "+":
                return a + b
            if k == "-":
                return a - b
            if k == "*":
                return a * b
            return a / b
        return ev(self.tree)

    def grad(self, p, f):
        """(g, [dg/dp_i for p_i in self.params]) by symbolic differentiation of
        the expression tree, evaluated at (p, f)."""
        idx = {name: i for i, name in enumerate(self.params)}
        m = len(self.params)

        def ev(n):
            k = n[0]
            if k == "num":
                return n[1], [0.0] * m
            if k == "feat":
                return f[n[1]], [0.0] * m
            if k == "par":
                d = [0.0] * m
                d[idx[n[1]]] = 1.0
                return p[n[1]], d
            if k == "neg":
                v, d = ev(n[1])
                return -v, [-x for x in d]
            if k == "fn":
                v, d = ev(n[2])
                if n[1] == "tanh":
                    y = math.tanh(v)
                    s = 1.0 - y * y
                elif n[1] == "exp":
                    y = math.exp(v)
                    s = y
                elif n[1] == "log":
                    y = math.log(v)
                    s = 1.0 / v
                else:
                    y = math.sqrt(v)
                    s = 0.5 / y
                return y, [s * x for x in d]
            a, da = ev(n[1])
            b, db = ev(n[2])
            if k == "+":
                return a + b, [x + y for x, y in zip(da, db)]
            if k == "-":
                return a - b, [x - y for x, y in zip(da, db)]
            if k == "*":
                return a * b, [x * b + a * y for x, y in zip(da, db)]
            return a / b, [(x * b - a * y) / (b * b) for x, y in zip(da, db)]
        return ev(self.tree)


def step_hat(x, p_edge):
    """Differentiable step of Section "Modeling Operation Overlap":
    s_hat(x) = (tanh(p_edge * x) + 1) / 2."""
    return (math.tanh(p_edge * x) + 1.0) / 2.0


def overlap_expr(c_overhead, c_gmem, c_onchip, edge="p_edge"):
    """Text of the nonlinear model of Section "Models Demonstrated":
    t = c_overhead + c_gmem * s_hat(c_gmem - c_onchip) + c_onchip * s_hat(c_onchip - c_gmem)."""
    g, o = "(%s)" % c_gmem, "(%s)" % c_onchip
    return "%s + %s * (tanh(%s * (%s - %s)) + 1) / 2 + %s * (tanh(%s * (%s - %s)) + 1) / 2" % (
        c_overhead, g, edge, g, o, o, edge, o, g)


def linear_expr(c_overhead, c_gmem, c_onchip):
    """Text of the linear model of Section "Models Demonstrated"."""
    return "%s + %s + %s" % (c_overhead, c_gmem, c_onchip)
