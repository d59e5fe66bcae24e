"""Expression trees and their FP64 evaluation (oracle; test infrastructure only).

Trees are written as S-expressions, e.g. the Sec. 4 style expression
``Z = A%B + 3.5*exp(C) - trans(D)`` is

    (- (+ (% A B) (* 3.5 (exp C))) (t D))

Operators (Sec. 4 expression suite and Sec. 3 functions):

    + - % /        element-wise; either operand may be a number (scalar op)
    *              number times matrix (scalar scale); matrix times matrix is
                   a matrix product, a fusion boundary
    neg exp log sqrt abs square sigmoid tanh      unary
    f32 X          X rounded to FP32 (round to nearest even): conv_to<fmat>
    pow X k        X to the number k;     gt X s   1 where X > s, else 0
    t X            transpose (Sec. 3: row and col swap before the access)
    each_col b     b (rows x 1) repeated over every column
    each_row b     b (1 x cols) repeated over every row
    accu E | sum E d | max E d | norm E           terminal reductions
                   (d = 0: one value per column, d = 1: one per row)

Leaves name matrices in ``env`` (``synth.Buffer``-like objects: ``data``,
``rows``, ``cols``, ``ld``, ``storage``). Element ``(r, c)`` of a leaf is
``data[r + c*ld]``, converted exactly to FP64 (Sec. 3, the element-access
rule for the base matrix type).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

import synth

from .sums import neumaier, neumaier_axis

BINARY = {"+", "-", "%", "/", "*"}
UNARY = {"neg", "exp", "log", "sqrt", "abs", "square", "sigmoid", "tanh", "f32"}
REDUCTIONS = {"accu", "sum", "max", "norm"}
_EXACT_UNARY = {"neg", "abs"}

_ARITY = {"neg": 1, "exp": 1, "log": 1, "sqrt": 1, "abs": 1, "square": 1, "sigmoid": 1,
          "tanh": 1, "f32": 1, "t": 1, "each_col": 1, "each_row": 1, "accu": 1, "norm": 1,
          "pow": 2, "gt": 2, "sum": 2, "max": 2, "+": 2, "-": 2, "%": 2, "/": 2, "*": 2}


@dataclasses.dataclass(eq=False)
class Node:
    op: str                       # "leaf", "num", or an operator
    args: list = dataclasses.field(default_factory=list)
    name: str | None = None       # leaf name
    value: float | None = None    # number

    def __repr__(self):
        if self.op == "leaf":
            return self.name
        if self.op == "num":
            return repr(self.value)
        return "(" + " ".join([self.op] + [repr(a) for a in self.args]) + ")"


def parse(text) -> Node:
    """S-expression -> Node tree (a Node is returned unchanged)."""
    if isinstance(text, Node):
        return text
    toks = text.replace("(", " ( ").replace(")", " ) ").split()
    pos = 0

    def atom(tok):
        try:
            return Node("num", value=float(tok))
        except ValueError:
            if not tok[0].isalpha():
                raise ValueError(f"bad atom {tok!r}")
            return Node("leaf", name=tok)

    def rec():
        nonlocal pos
        tok = toks[pos]
        pos += 1
        if tok == "(":
            op = toks[pos]
            pos += 1
            args = []
            while toks[pos] != ")":
                args.append(rec())
            pos += 1
            return Node(op, args)
        if tok == ")":
            raise ValueError("unbalanced ')'")
        return atom(tok)

    node = rec()
    if pos != len(toks):
        raise ValueError("trailing tokens")
    _check_arity(node)
    return node


def _check_arity(n: Node):
    if n.op in ("leaf", "num"):
        return
    if n.op not in _ARITY:
        raise ValueError(f"unknown operator {n.op!r}")
    if len(n.args) != _ARITY[n.op]:
        raise ValueError(f"{n.op} takes {_ARITY[n.op]} operands")
    for a in n.args:
        _check_arity(a)


def leaves_of(node) -> list:
    """Leaf names, first occurrence order."""
    out = []

    def rec(n):
        if n.op == "leaf" and n.name not in out:
            out.append(n.name)
        for a in n.args:
            rec(a)

    rec(parse(node))
    return out


def _is_product(n: Node) -> bool:
    return n.op == "*" and n.args[0].op != "num" and n.args[1].op != "num"


# ---------------------------------------------------------------- shapes

def shape_of(node, env) -> tuple | None:
    """Logical shape; ``None`` for a number. Broadcast nodes report
    ``("col", rows)`` / ``("row", cols)``."""
    n = parse(node)
    op = n.op
    if op == "num":
        return None
    if op == "leaf":
        b = env[n.name]
        return (b.rows, b.cols)
    if op == "t":
        s = shape_of(n.args[0], env)
        return (s[1], s[0])
    if op == "each_col":
        r, c = shape_of(n.args[0], env)
        if c != 1:
            raise ValueError("each_col needs a column vector")
        return ("col", r)
    if op == "each_row":
        r, c = shape_of(n.args[0], env)
        if r != 1:
            raise ValueError("each_row needs a row vector")
        return ("row", c)
    if op in UNARY or op in ("pow", "gt"):
        s = shape_of(n.args[0], env)
        if s is None or isinstance(s[0], str):
            raise ValueError(f"{op} needs a matrix operand")
        return s
    if op in BINARY:
        a, b = (shape_of(x, env) for x in n.args)
        if _is_product(n):
            if a[1] != b[0]:
                raise ValueError("matrix product: inner sizes differ")
            return (a[0], b[1])
        if a is None and b is None:
            raise ValueError("two numbers")
        if a is None or b is None:
            s = a if b is None else b
            if isinstance(s[0], str):
                raise ValueError("a broadcast needs a matrix partner")
            return s
        return _bcast_shape(a, b)
    if op in REDUCTIONS:
        r, c = shape_of(n.args[0], env)
        if op in ("accu", "norm"):
            return (1, 1)
        d = int(n.args[1].value)
        if d not in (0, 1):
            raise ValueError("dimension must be 0 or 1")
        return (1, c) if d == 0 else (r, 1)
    raise ValueError(op)


def _bcast_shape(a, b):
    if isinstance(a[0], str) and isinstance(b[0], str):
        raise ValueError("two broadcasts")
    if isinstance(b[0], str):
        a, b = b, a
    if isinstance(a[0], str):
        kind, n = a
        if (kind == "col" and b[0] != n) or (kind == "row" and b[1] != n):
            raise ValueError("broadcast size mismatch")
        return b
    if a != b:
        raise ValueError(f"shape mismatch {a} vs {b}")
    return a


# ---------------------------------------------------------------- element values

def _leaf_values(buf, R, C):
    """Sec. 3 base rule: element (row, col) is in[row + col*ld]."""
    R = np.asarray(R, dtype=np.int64)
    C = np.asarray(C, dtype=np.int64)
    if np.any(R < 0) or np.any(R >= buf.rows) or np.any(C < 0) or np.any(C >= buf.cols):
        raise IndexError("leaf access out of range")
    return synth.to_f64(buf.data[R + C * buf.ld], buf.storage)


def _apply_unary(op, a):
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        if op == "neg":
            return -a
        if op == "exp":
            return np.exp(a)
        if op == "log":
            return np.log(a)
        if op == "sqrt":
            return np.sqrt(a)
        if op == "abs":
            return np.abs(a)
        if op == "square":
            return a * a
        if op == "sigmoid":                      # Sec. 4: 1 / (1 + exp(-X))
            return 1.0 / (1.0 + np.exp(-a))
        if op == "tanh":
            return np.tanh(a)
        if op == "f32":                          # Sec. 4 expr3: conv_to<fmat>, round to nearest
            return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)
    raise ValueError(op)


def _unary_deriv(op, a, z):
    """d op(a) / da, given a and z = op(a)."""
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        if op == "neg":
            return -np.ones_like(a)
        if op == "exp":
            return z
        if op == "log":
            return 1.0 / a
        if op == "sqrt":
            return 0.5 / z
        if op == "abs":
            return np.sign(a)
        if op == "square":
            return 2.0 * a
        if op == "sigmoid":
            return z * (1.0 - z)
        if op == "tanh":
            return 1.0 - z * z
        if op == "f32":
            return np.ones_like(a)
    raise ValueError(op)


def _binary(op, a, b):
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        if op == "+":
            return a + b
        if op == "-":
            return a - b
        if op in ("%", "*"):
            return a * b
        if op == "/":
            return a / b
    raise ValueError(op)


def _materialise(n: Node, env):
    r, c = shape_of(n, env)
    return np.broadcast_to(at(n, env, np.arange(r)[:, None], np.arange(c)[None, :]), (r, c))


def _materialise_sigma(n: Node, env):
    r, c = shape_of(n, env)
    v, sg = at_sigma(n, env, np.arange(r)[:, None], np.arange(c)[None, :])
    return np.broadcast_to(v, (r, c)), np.broadcast_to(sg, (r, c))


def at(node, env, R, C):
    """Values of an element-wise tree at positions ``(R, C)`` of its logical
    matrix (``R``, ``C`` broadcastable integer index arrays).

    This is the recursive element-access rule of Sec. 3: a leaf reads
    ``in[row + col*ld]``; ``t`` swaps row and col for its operand; a scalar
    node wraps its operand's access; ``each_col b`` reads ``b(row, 0)`` and
    ``each_row b`` reads ``b(0, col)``.
    """
    n = parse(node)
    op = n.op
    if op == "num":
        return n.value
    if op == "leaf":
        return _leaf_values(env[n.name], R, C)
    if op == "t":
        return at(n.args[0], env, C, R)
    if op == "each_col":
        return at(n.args[0], env, R, np.zeros_like(np.asarray(C)))
    if op == "each_row":
        return at(n.args[0], env, np.zeros_like(np.asarray(R)), C)
    if op in UNARY:
        return _apply_unary(op, at(n.args[0], env, R, C))
    if op == "pow":
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
            return np.power(at(n.args[0], env, R, C), n.args[1].value)
    if op == "gt":
        return (at(n.args[0], env, R, C) > n.args[1].value).astype(np.float64)
    if _is_product(n):
        # matrix product: a fusion boundary; both operands are materialised
        prod = _materialise(n.args[0], env) @ _materialise(n.args[1], env)
        return prod[np.asarray(R), np.asarray(C)]
    if op in BINARY:
        return _binary(op, at(n.args[0], env, R, C), at(n.args[1], env, R, C))
    raise ValueError(f"{op} is not element-wise")


def at_sigma(node, env, R, C):
    """``(value, sigma)`` at positions ``(R, C)``.

    ``sigma`` is a first-order running error bound in units of the unit
    roundoff: evaluating the tree with rounding ``u`` per operation gives an
    error of at most about ``k*u*sigma`` (``k`` a small constant). Leaves
    and numbers are exact (``sigma = 0``); every operation adds the rounding
    of its own result (``|z|``) to the propagated errors of its operands:

        z = a +- b    sigma_a + sigma_b + |z|
        z = a % b     sigma_a|b| + sigma_b|a| + |z|
        z = a / b     (sigma_a + |z| sigma_b) / |b| + |z|
        z = f(a)      |f'(a)| sigma_a + |z|   (no |z| for neg and abs: exact)
        z = t(a), broadcasts: sigma of the operand at the mapped position
    """
    n = parse(node)
    op = n.op
    if op == "num":
        return n.value, 0.0
    if op == "leaf":
        v = _leaf_values(env[n.name], R, C)
        return v, np.zeros_like(v)
    if op == "t":
        return at_sigma(n.args[0], env, C, R)
    if op == "each_col":
        return at_sigma(n.args[0], env, R, np.zeros_like(np.asarray(C)))
    if op == "each_row":
        return at_sigma(n.args[0], env, np.zeros_like(np.asarray(R)), C)
    if op in UNARY:
        a, sa = at_sigma(n.args[0], env, R, C)
        z = _apply_unary(op, a)
        with np.errstate(invalid="ignore", over="ignore"):
            d = np.where(sa == 0, 0.0, np.abs(_unary_deriv(op, a, z)) * sa)
        if op in _EXACT_UNARY:
            return z, d
        return z, d + np.abs(z)
    if op == "pow":
        a, sa = at_sigma(n.args[0], env, R, C)
        k = n.args[1].value
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
            z = np.power(a, k)
            d = np.where(sa == 0, 0.0, np.abs(k * np.power(a, k - 1)) * sa)
        return z, d + np.abs(z)
    if op == "gt":
        a, _ = at_sigma(n.args[0], env, R, C)
        z = (a > n.args[1].value).astype(np.float64)
        return z, np.zeros_like(z)
    if _is_product(n):
        # dot products of length K summed in order: the standard forward
        # bound |fl(x.y) - x.y| <= K u |x|.|y| (Higham, Accuracy and
        # Stability of Numerical Algorithms, Sec. 3.1), plus the operands'
        # own errors carried through the products
        A, sA = _materialise_sigma(n.args[0], env)
        B, sB = _materialise_sigma(n.args[1], env)
        K = A.shape[1]
        z = A @ B
        s = sA @ np.abs(B) + np.abs(A) @ sB + K * (np.abs(A) @ np.abs(B))
        R, C = np.broadcast_arrays(np.asarray(R), np.asarray(C))
        return z[R, C], s[R, C]
    if op in BINARY:
        a, sa = at_sigma(n.args[0], env, R, C)
        b, sb = at_sigma(n.args[1], env, R, C)
        z = _binary(op, a, b)
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
            if op in ("+", "-"):
                s = sa + sb + np.abs(z)
            elif op in ("%", "*"):
                s = sa * np.abs(b) + sb * np.abs(a) + np.abs(z)
            else:
                s = (sa + np.abs(z) * sb) / np.abs(b) + np.abs(z)
        return z, s
    raise ValueError(f"{op} is not element-wise")


def at_mag(node, env, R, C):
    """Magnitude scale ``m`` at positions ``(R, C)``: the tree evaluated on
    absolute values, with every sign-dependent step made sign-free.

        m(leaf) = |leaf|           m(number) = |number|
        m(a +- b) = m(a) + m(b)    m(a % b) = m(a) m(b)   m(a / b) = m(a) / |b|
        m(f(a)) = |f(m(a))| for the unary functions (neg and abs: m(a))
        m(pow(a, k)) = m(a)^k      m(gt(a, s)) = gt(a, s) (exact 0 or 1)
        m(matrix product) = |A| |B| (products of magnitudes, summed)
        t and broadcasts map positions as the value rule does

    For trees of sums, differences, products, quotients and scalars of
    exactly stored leaves this is the componentwise condition scale of
    rounding-error analysis (Higham, Accuracy and Stability of Numerical
    Algorithms, Sec. 3.1-3.3): evaluating such a tree with unit roundoff u
    errs by at most about k u m for a small k set by the tree's depth, and
    m >= |value|. Transcendental nodes carry no such bound (an error in
    their argument is amplified by the derivative), which is why at_sigma
    exists; m is the scale for the trees without them.
    """
    n = parse(node)
    op = n.op
    if op == "num":
        return abs(n.value)
    if op == "leaf":
        return np.abs(_leaf_values(env[n.name], R, C))
    if op == "t":
        return at_mag(n.args[0], env, C, R)
    if op == "each_col":
        return at_mag(n.args[0], env, R, np.zeros_like(np.asarray(C)))
    if op == "each_row":
        return at_mag(n.args[0], env, np.zeros_like(np.asarray(R)), C)
    if op in UNARY:
        a = at_mag(n.args[0], env, R, C)
        if op in _EXACT_UNARY:
            return a
        return np.abs(_apply_unary(op, a))
    if op == "pow":
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
            return np.abs(np.power(at_mag(n.args[0], env, R, C), n.args[1].value))
    if op == "gt":
        return at(n, env, R, C)
    if _is_product(n):
        A = np.abs(_materialise(n.args[0], env))
        B = np.abs(_materialise(n.args[1], env))
        R, C = np.broadcast_arrays(np.asarray(R), np.asarray(C))
        return (A @ B)[R, C]
    if op in BINARY:
        a = at_mag(n.args[0], env, R, C)
        b = at_mag(n.args[1], env, R, C)
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
            if op in ("+", "-"):
                return a + b
            if op in ("%", "*"):
                return a * b
            return a / np.abs(at(n.args[1], env, R, C))
    raise ValueError(f"{op} is not element-wise")


def evaluate_mag(node, env) -> np.ndarray:
    """Magnitude scale of a whole result (same shape as ``evaluate``): the
    element-wise ``at_mag``; a sum (accu, sum along a dimension) sums the
    magnitudes of its terms; max takes the largest magnitude of the slice;
    norm is the 2-norm of the magnitudes."""
    n = parse(node)
    if n.op not in REDUCTIONS:
        r, c = shape_of(n, env)
        out = np.empty((r, c))
        for c0, c1 in _panels(r, c):
            out[:, c0:c1] = np.broadcast_to(
                at_mag(n, env, np.arange(r)[:, None], np.arange(c0, c1)[None, :]), (r, c1 - c0))
        return out
    inner = n.args[0]
    r, c = shape_of(inner, env)
    if n.op in ("accu", "norm"):
        state = None
        for c0, c1 in _panels(r, c):
            m = np.broadcast_to(at_mag(inner, env, np.arange(r)[:, None],
                                       np.arange(c0, c1)[None, :]), (r, c1 - c0))
            state = neumaier_axis(m * m if n.op == "norm" else m, axis=1, state=state)
        tot = _combine(*state) if state is not None else 0.0
        return np.array([[math.sqrt(tot) if n.op == "norm" else tot]])
    d = int(n.args[1].value)
    out = np.zeros((1, c)) if d == 0 else np.zeros((r, 1))
    for c0, c1 in _panels(r, c):
        m = np.broadcast_to(at_mag(inner, env, np.arange(r)[:, None], np.arange(c0, c1)[None, :]),
                            (r, c1 - c0))
        if d == 0:
            out[0, c0:c1] = np.max(m, axis=0) if n.op == "max" else np.sum(m, axis=0)
        elif n.op == "max":
            out[:, 0] = np.maximum(out[:, 0], np.max(m, axis=1))
        else:
            out[:, 0] += np.sum(m, axis=1)
    return out


# ---------------------------------------------------------------- whole results

def _panels(rows, cols, budget=1 << 23):
    w = max(1, budget // max(rows, 1))
    for c0 in range(0, cols, w):
        yield c0, min(cols, c0 + w)


def _element_panels(node, env, with_sigma):
    """Column panels of an element-wise tree: ``(c0, c1, value, sigma)``."""
    r, c = shape_of(node, env)
    for c0, c1 in _panels(r, c):
        R = np.arange(r)[:, None]
        C = np.arange(c0, c1)[None, :]
        if with_sigma:
            v, s = at_sigma(node, env, R, C)
            yield c0, c1, np.broadcast_to(v, (r, c1 - c0)), np.broadcast_to(s, (r, c1 - c0))
        else:
            yield c0, c1, np.broadcast_to(at(node, env, R, C), (r, c1 - c0)), None


def evaluate(node, env) -> np.ndarray:
    """The expression's value as an FP64 matrix (1x1 for accu and norm)."""
    return _evaluate(parse(node), env, with_sigma=False)[0]


def evaluate_sigma(node, env):
    """``(value, sigma)`` as FP64 matrices; see ``at_sigma`` for sigma."""
    return _evaluate(parse(node), env, with_sigma=True)


def _combine(part_s, part_c) -> float:
    """Compensated sum of per-row (sum, correction) pairs, in row order."""
    pairs = np.stack([np.asarray(part_s), np.asarray(part_c)], axis=1).ravel()
    return neumaier(pairs)


def _evaluate(n: Node, env, with_sigma):
    if n.op not in REDUCTIONS:
        r, c = shape_of(n, env)
        out = np.empty((r, c))
        sig = np.empty((r, c)) if with_sigma else None
        for c0, c1, v, s in _element_panels(n, env, with_sigma):
            out[:, c0:c1] = v
            if with_sigma:
                sig[:, c0:c1] = s
        return out, sig
    inner = n.args[0]
    if n.op in ("accu", "norm"):
        return _full_reduction(n.op, inner, env, with_sigma)
    d = int(n.args[1].value)
    if n.op == "sum":
        return _sum_dim(inner, d, env, with_sigma)
    return _max_dim(inner, d, env, with_sigma)


def _full_reduction(op, inner, env, with_sigma):
    """accu: the sum of every element. norm: the square root of the sum of
    squares (the vectorised 2-norm, i.e. the Frobenius norm of a matrix).
    Each row is summed across the columns, panel after panel, then the row
    sums are summed; every sum is compensated."""
    state = None
    sstate = None
    for _, _, v, s in _element_panels(inner, env, with_sigma):
        term = v * v if op == "norm" else v
        state = neumaier_axis(term, axis=1, state=state)
        if with_sigma:
            # sigma of v*v is 2|v|sigma_v + v^2; a sum adds sum|term|
            st = (2.0 * np.abs(v) * s + 2.0 * term) if op == "norm" else (s + np.abs(v))
            sstate = neumaier_axis(st, axis=1, state=sstate)
    total = _combine(*state)
    sig = None
    if with_sigma:
        stot = _combine(*sstate)
        if op == "norm":
            nv = math.sqrt(total)
            sig = np.array([[stot / (2.0 * nv) + nv if nv > 0 else 0.0]])
        else:
            sig = np.array([[stot]])
    val = math.sqrt(total) if op == "norm" else total
    return np.array([[val]]), sig


def _sum_dim(inner, d, env, with_sigma):
    """sum(E, 0): one compensated sum per column; sum(E, 1): one per row."""
    r, c = shape_of(inner, env)
    if d == 0:
        out = np.empty((1, c))
        sig = np.empty((1, c)) if with_sigma else None
        for c0, c1, v, s in _element_panels(inner, env, with_sigma):
            cs, cc = neumaier_axis(v, axis=0)
            out[0, c0:c1] = cs + cc
            if with_sigma:
                ss, sc = neumaier_axis(s + np.abs(v), axis=0)
                sig[0, c0:c1] = ss + sc
        return out, sig
    state = None
    sstate = None
    for _, _, v, s in _element_panels(inner, env, with_sigma):
        state = neumaier_axis(v, axis=1, state=state)
        if with_sigma:
            sstate = neumaier_axis(s + np.abs(v), axis=1, state=sstate)
    out = (state[0] + state[1])[:, None]
    sig = (sstate[0] + sstate[1])[:, None] if with_sigma else None
    return out, sig


def _max_dim(inner, d, env, with_sigma):
    """max(E, 0): per column; max(E, 1): per row. NaN propagates
    (``np.max`` and ``np.maximum`` propagate it). The error of a max of
    computed values is at most the largest error among them, so sigma is
    the largest sigma of the slice."""
    r, c = shape_of(inner, env)
    if d == 0:
        out = np.empty((1, c))
        sig = np.empty((1, c)) if with_sigma else None
        for c0, c1, v, s in _element_panels(inner, env, with_sigma):
            out[0, c0:c1] = np.max(v, axis=0)
            if with_sigma:
                sig[0, c0:c1] = np.max(s, axis=0)
        return out, sig
    out = None
    sig = None
    for _, _, v, s in _element_panels(inner, env, with_sigma):
        m = np.max(v, axis=1)
        out = m if out is None else np.maximum(out, m)
        if with_sigma:
            ms = np.max(s, axis=1)
            sig = ms if sig is None else np.maximum(sig, ms)
    return out[:, None], (sig[:, None] if with_sigma else None)
