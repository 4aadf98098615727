"""Symbolic dispersion relations: an expression graph that differentiates and
simplifies itself and emits the fused CUDA evaluator of D and its gradients.

This is the front end the paper is built around (Sec. 2): expressions are
trees of nodes built by factory functions that consult a cache keyed by the
sub-graph's structure, so an identical sub-graph is created once (Sec. 2.1);
every factory applies simplification rules as the node is built ("reduce":
constant folding, x + 0, x * 1, x * 0, collection of constant factors and of
repeated terms); ``df`` applies the chain rule node by node, with constants
differentiating to zero and variables to one or zero (Sec. 2.1).  Code
generation walks the graph from the outputs, gives every node one register
and emits each shared sub-graph once (Sec. 2.2).  The emitted function is
compiled at run time by the library (``gf_jit_medium_create``) into an RK4
ray kernel for sm_103a.

Variables: x0, x1, x2 (position), k0, k1, k2 (wave vector), w (frequency).
"""
from __future__ import annotations

import math
import numpy as np

# ------------------------------------------------------------------ the graph

_CACHE: dict[tuple, "Node"] = {}
_NEXT_ID = [0]

VARS = ("x0", "x1", "x2", "k0", "k1", "k2", "w")


class Node:
    """One node of the expression graph (immutable, hash-consed)."""

    __slots__ = ("op", "args", "value", "id")

    def __init__(self, op: str, args: tuple, value):
        self.op = op
        self.args = args
        self.value = value
        self.id = _NEXT_ID[0]
        _NEXT_ID[0] += 1

    # operator overloading builds graph nodes (Sec. 2.1)
    def __add__(self, o): return add(self, lift(o))
    def __radd__(self, o): return add(lift(o), self)
    def __sub__(self, o): return add(self, neg(lift(o)))
    def __rsub__(self, o): return add(lift(o), neg(self))
    def __mul__(self, o): return mul(self, lift(o))
    def __rmul__(self, o): return mul(lift(o), self)
    def __truediv__(self, o): return mul(self, inv(lift(o)))
    def __rtruediv__(self, o): return mul(lift(o), inv(self))
    def __neg__(self): return neg(self)

    def __pow__(self, n):
        if not isinstance(n, int):
            raise TypeError("only integer powers")
        return power(self, n)

    def __repr__(self):
        return to_str(self)

    @property
    def is_const(self) -> bool:
        return self.op == "const"


def _make(op: str, args: tuple, value=None) -> Node:
    key = (op, tuple(a.id for a in args), value)
    node = _CACHE.get(key)
    if node is None:
        node = Node(op, args, value)
        _CACHE[key] = node
    return node


def cache_size() -> int:
    return len(_CACHE)


def const(v: float) -> Node:
    v = float(v)
    if v == 0.0:
        v = 0.0          # one zero (no -0.0 node)
    return _make("const", (), v)


def var(name: str) -> Node:
    if name not in VARS:
        raise ValueError(f"unknown variable {name}")
    return _make("var", (), name)


def lift(v) -> Node:
    return v if isinstance(v, Node) else const(v)


ZERO = const(0.0)
ONE = const(1.0)


def _split_coeff(n: Node) -> tuple[float, Node]:
    """n = c * rest with a constant factor c pulled out."""
    if n.op == "mul" and n.args[0].is_const:
        return n.args[0].value, n.args[1]
    if n.op == "neg":
        c, r = _split_coeff(n.args[0])
        return -c, r
    return 1.0, n


def add(a: Node, b: Node) -> Node:
    if a.is_const and b.is_const:
        return const(a.value + b.value)
    if a.is_const and a.value == 0.0:
        return b
    if b.is_const and b.value == 0.0:
        return a
    ca, ra = _split_coeff(a)
    cb, rb = _split_coeff(b)
    if ra is rb and not ra.is_const:           # c1 x + c2 x -> (c1 + c2) x
        return mul(const(ca + cb), ra)
    if b.is_const and not a.is_const:           # constants first
        a, b = b, a
    elif not a.is_const and not b.is_const and b.id < a.id:
        a, b = b, a                             # canonical order of a commutative op
    return _make("add", (a, b))


def mul(a: Node, b: Node) -> Node:
    if a.is_const and b.is_const:
        return const(a.value * b.value)
    if b.is_const:
        a, b = b, a
    if a.is_const:
        if a.value == 0.0:
            return ZERO
        if a.value == 1.0:
            return b
        if a.value == -1.0:
            return neg(b)
        if b.op == "mul" and b.args[0].is_const:            # c1 (c2 x) -> (c1 c2) x
            return mul(const(a.value * b.args[0].value), b.args[1])
        if b.op == "neg":
            return mul(const(-a.value), b.args[0])
        return _make("mul", (a, b))
    if a.op == "neg" or b.op == "neg":                       # (-x) y -> -(x y)
        x = a.args[0] if a.op == "neg" else a
        y = b.args[0] if b.op == "neg" else b
        r = mul(x, y)
        return r if (a.op == "neg") == (b.op == "neg") else neg(r)
    if a.op == "mul" and a.args[0].is_const:                 # (c x) y -> c (x y)
        return mul(a.args[0], mul(a.args[1], b))
    if b.op == "mul" and b.args[0].is_const:
        return mul(b.args[0], mul(a, b.args[1]))
    if a is b:
        return power(a, 2)
    if b.id < a.id:
        a, b = b, a
    return _make("mul", (a, b))


def neg(a: Node) -> Node:
    if a.is_const:
        return const(-a.value)
    if a.op == "neg":
        return a.args[0]
    if a.op == "mul" and a.args[0].is_const:
        return mul(const(-a.args[0].value), a.args[1])
    return _make("neg", (a,))


def inv(a: Node) -> Node:
    if a.is_const:
        if a.value == 0.0:
            raise ZeroDivisionError("1/0 in an expression")
        return const(1.0 / a.value)
    if a.op == "inv":
        return a.args[0]
    return _make("inv", (a,))


def power(a: Node, n: int) -> Node:
    if n == 0:
        return ONE
    if n == 1:
        return a
    if a.is_const:
        return const(a.value ** n)
    if n < 0:
        return inv(power(a, -n))
    if a.op == "pow":
        return power(a.args[0], a.value * n)
    return _make("pow", (a,), n)


def exp(a: Node) -> Node:
    a = lift(a)
    if a.is_const:
        return const(math.exp(a.value))
    return _make("exp", (a,))


def sqrt(a: Node) -> Node:
    a = lift(a)
    if a.is_const:
        return const(math.sqrt(a.value))
    return _make("sqrt", (a,))


def where_nonpos(c: Node, a: Node, b: Node) -> Node:
    """a where c <= 0, else b (piecewise definitions, e.g. inside a lens)."""
    c, a, b = lift(c), lift(a), lift(b)
    if c.is_const:
        return a if c.value <= 0.0 else b
    if a is b:
        return a
    return _make("where", (c, a, b))


# ------------------------------------------------------------------ calculus

_DF_CACHE: dict[tuple[int, str], Node] = {}


def df(n: Node, v: str) -> Node:
    """d n / d v by the chain rule (memoised per node and variable)."""
    key = (n.id, v)
    r = _DF_CACHE.get(key)
    if r is not None:
        return r
    op = n.op
    if op == "const":
        r = ZERO
    elif op == "var":
        r = ONE if n.value == v else ZERO
    elif op == "add":
        r = add(df(n.args[0], v), df(n.args[1], v))
    elif op == "mul":
        a, b = n.args
        r = add(mul(df(a, v), b), mul(a, df(b, v)))
    elif op == "neg":
        r = neg(df(n.args[0], v))
    elif op == "inv":
        r = neg(mul(power(n, 2), df(n.args[0], v)))
    elif op == "pow":
        a = n.args[0]
        r = mul(mul(const(n.value), power(a, n.value - 1)), df(a, v))
    elif op == "exp":
        r = mul(n, df(n.args[0], v))
    elif op == "sqrt":
        r = mul(mul(const(0.5), inv(n)), df(n.args[0], v))
    elif op == "where":
        c, a, b = n.args
        r = where_nonpos(c, df(a, v), df(b, v))
    else:
        raise ValueError(op)
    _DF_CACHE[key] = r
    return r


def gradients(D: Node) -> list[Node]:
    """[D, D_x0, D_x1, D_x2, D_k0, D_k1, D_k2, D_w]."""
    return [D] + [df(D, v) for v in ("x0", "x1", "x2", "k0", "k1", "k2", "w")]


# ------------------------------------------------------------------ evaluation

def evaluate(outs: list[Node], env: dict[str, np.ndarray]) -> list[np.ndarray]:
    """Evaluate nodes with numpy arrays bound to the variables (for tests)."""
    memo: dict[int, np.ndarray] = {}

    def ev(n: Node):
        r = memo.get(n.id)
        if r is not None:
            return r
        op = n.op
        if op == "const":
            r = n.value
        elif op == "var":
            r = env[n.value]
        elif op == "add":
            r = ev(n.args[0]) + ev(n.args[1])
        elif op == "mul":
            r = ev(n.args[0]) * ev(n.args[1])
        elif op == "neg":
            r = -ev(n.args[0])
        elif op == "inv":
            r = 1.0 / ev(n.args[0])
        elif op == "pow":
            r = ev(n.args[0]) ** n.value
        elif op == "exp":
            r = np.exp(ev(n.args[0]))
        elif op == "sqrt":
            r = np.sqrt(ev(n.args[0]))
        elif op == "where":
            r = np.where(ev(n.args[0]) <= 0.0, ev(n.args[1]), ev(n.args[2]))
        memo[n.id] = r
        return r

    return [np.broadcast_to(ev(o), np.broadcast(*env.values()).shape).copy() for o in outs]


def to_str(n: Node) -> str:
    op = n.op
    if op == "const":
        return repr(n.value)
    if op == "var":
        return n.value
    if op == "add":
        return f"({to_str(n.args[0])} + {to_str(n.args[1])})"
    if op == "mul":
        return f"{to_str(n.args[0])}*{to_str(n.args[1])}"
    if op == "neg":
        return f"-({to_str(n.args[0])})"
    if op == "inv":
        return f"1/({to_str(n.args[0])})"
    if op == "pow":
        return f"({to_str(n.args[0])})^{n.value}"
    if op in ("exp", "sqrt"):
        return f"{op}({to_str(n.args[0])})"
    if op == "where":
        return f"where({to_str(n.args[0])} <= 0, {to_str(n.args[1])}, {to_str(n.args[2])})"
    return op


def count_nodes(outs: list[Node]) -> int:
    seen: set[int] = set()
    stack = list(outs)
    while stack:
        n = stack.pop()
        if n.id in seen:
            continue
        seen.add(n.id)
        stack.extend(n.args)
    return len(seen)


# ------------------------------------------------------------------ code generation

def _lit(v: float) -> str:
    if math.isinf(v) or math.isnan(v):
        raise ValueError("non-finite constant in an expression")
    return float.hex(v)


def to_cuda(outs: list[Node], name: str = "gf_user_dispersion") -> str:
    """CUDA source of a device function computing the outputs from
    y = (x0, x1, x2, k0, k1, k2) and w into out[0..len(outs)): one register per
    node in topological order, every shared sub-graph emitted once."""
    order: list[Node] = []
    seen: set[int] = set()

    def visit(n: Node):
        stack = [(n, False)]
        while stack:
            m, done = stack.pop()
            if done:
                order.append(m)
                continue
            if m.id in seen:
                continue
            seen.add(m.id)
            stack.append((m, True))
            for a in reversed(m.args):
                if a.id not in seen:
                    stack.append((a, False))

    for o in outs:
        visit(o)
    ref: dict[int, str] = {}
    lines = []
    inputs = {"x0": "y[0]", "x1": "y[1]", "x2": "y[2]", "k0": "y[3]", "k1": "y[4]", "k2": "y[5]", "w": "w"}
    for n in order:
        op = n.op
        if op == "const":
            ref[n.id] = _lit(n.value)
            continue
        if op == "var":
            ref[n.id] = inputs[n.value]
            continue
        a = [ref[x.id] for x in n.args]
        if op == "add":
            e = f"{a[0]} + {a[1]}"
        elif op == "mul":
            e = f"{a[0]} * {a[1]}"
        elif op == "neg":
            e = f"-{a[0]}"
        elif op == "inv":
            e = f"1.0 / {a[0]}"
        elif op == "pow":
            e = " * ".join([a[0]] * n.value)
        elif op == "exp":
            e = f"gf_exp({a[0]})"
        elif op == "sqrt":
            e = f"sqrt({a[0]})"
        elif op == "where":
            e = f"({a[0]} <= 0.0) ? {a[1]} : {a[2]}"
        else:
            raise ValueError(op)
        ref[n.id] = f"v{n.id}"
        lines.append(f"    const double v{n.id} = {e};")
    body = "\n".join(lines)
    assigns = "\n".join(f"    out[{i}] = {ref[o.id]};" for i, o in enumerate(outs))
    return (f"__device__ __forceinline__ void {name}(const double *__restrict__ y, const double w,\n"
            f"                                         double *__restrict__ out)\n{{\n{body}\n{assigns}\n}}\n")


# ------------------------------------------------------------------ media

def x():
    return var("x0"), var("x1"), var("x2")


def k():
    return var("k0"), var("k1"), var("k2")


def isotropic(n2: Node) -> Node:
    """D = |k|^2 - w^2 n^2(x)."""
    k0, k1, k2 = k()
    w = var("w")
    return k0 ** 2 + k1 ** 2 + k2 ** 2 - w ** 2 * n2


def gaussian_blobs(blobs) -> Node:
    """sum_j A_j exp(-|x - c_j|^2 / (2 w_j^2)) from rows (A, cx, cy, cz, w)."""
    x0, x1, x2 = x()
    total = ZERO
    for A, cx, cy, cz, wj in np.asarray(blobs, dtype=np.float64).reshape(-1, 5):
        q = (x0 - cx) ** 2 + (x1 - cy) ** 2 + (x2 - cz) ** 2
        total = total + A * exp(q * (-1.0 / (2.0 * wj * wj)))
    return total


def grin_n2(n0: float, a: float) -> Node:
    x0, x1, x2 = x()
    return n0 * n0 * (1.0 - a * a * (x1 ** 2 + x2 ** 2))


def luneburg_n2() -> Node:
    x0, x1, x2 = x()
    r2 = x0 ** 2 + x1 ** 2 + x2 ** 2
    return where_nonpos(r2 - 1.0, 2.0 - r2, ONE)


def medium_source(D: Node, name: str = "gf_user_dispersion") -> str:
    """Generated CUDA for D and its seven partial derivatives."""
    return to_cuda(gradients(D), name)


def cold_plasma(species, profile=(1.0, 0.0, 1.0, 0.0)) -> Node:
    """Cold magnetised plasma, B along z (Sec. 4.1, Eqs. 5-10), built from its
    definition: S, Dst and P from the species' plasma and cyclotron
    frequencies, w_p^2 (f0 + f1 x0) and Omega (g0 + g1 x0), n = k / w, and
    D = det(eps + n n - n^2 I) in the Stix form; the gradients come from df."""
    x0, _, _ = x()
    k0, k1, k2 = k()
    w = var("w")
    f0, f1, g0, g1 = profile
    f = f0 + f1 * x0
    g = g0 + g1 * x0
    S_, Dst, P = ONE, ZERO, ONE
    for wp2, om in species:
        wp = wp2 * f
        W = om * g
        den = w ** 2 - W ** 2
        S_ = S_ - wp / den
        Dst = Dst + W * wp / (w * den)
        P = P - wp / w ** 2
    a = (k0 ** 2 + k1 ** 2) / w ** 2
    b = k2 ** 2 / w ** 2
    RL = S_ ** 2 - Dst ** 2
    return S_ * a * (a + b) + P * b * (a + b) - RL * a - P * S_ * (a + 2.0 * b) + P * RL
