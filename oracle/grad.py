"""Reverse-mode gradient of L = accu(f(leaves)) (oracle; test infrastructure only).

``L`` is the sum of ``f`` over every output element, so the derivative of
``L`` with respect to one stored leaf element is the sum, over the output
elements whose evaluation reads it, of the local partial derivative of
``f`` there. The local partials come from the textbook reverse pass over
the tree (adjoint of the root is ``gL``; each node hands its adjoint to its
operands times its partial derivative); the sum over readers is the adjoint
of the gather in the Sec. 3 element-access rule: a scatter-add at the same
positions ``row + col*ld`` that the forward pass read.

Derivative rules (z = node value, a, b operands, s a number):

    a + b -> (1, 1)        a - b -> (1, -1)        a % b -> (b, a)
    a / b -> (1/b, -a/b^2) s * a -> s              neg -> -1
    exp -> z   log -> 1/a  sqrt -> 1/(2z)  abs -> sign(a)  square -> 2a
    sigmoid -> z(1 - z)    tanh -> 1 - z^2         pow(a, k) -> k a^(k-1)
    gt(a, s) -> 0 (piecewise constant)
    t: the operand's element (col, row); each_col b: b(row, 0); each_row b: b(0, col)
"""
from __future__ import annotations

import numpy as np

from .expr import parse, at, shape_of, _unary_deriv, _apply_unary, _is_product, UNARY


def _backprop(n, env, R, C, adj, out):
    op = n.op
    if op == "num":
        return
    if op == "leaf":
        out.append((n.name, R, C, adj))
        return
    if op == "t":
        _backprop(n.args[0], env, C, R, adj, out)
        return
    if op == "each_col":
        _backprop(n.args[0], env, R, np.zeros_like(np.asarray(C)), adj, out)
        return
    if op == "each_row":
        _backprop(n.args[0], env, np.zeros_like(np.asarray(R)), C, adj, out)
        return
    if op in UNARY:
        a = at(n.args[0], env, R, C)
        z = _apply_unary(op, a)
        _backprop(n.args[0], env, R, C, adj * _unary_deriv(op, a, z), out)
        return
    if op == "pow":
        a = at(n.args[0], env, R, C)
        k = n.args[1].value
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
            _backprop(n.args[0], env, R, C, adj * k * np.power(a, k - 1), out)
        return
    if op == "gt":
        return
    if _is_product(n):
        raise ValueError("no fused gradient through a matrix product")
    x, y = n.args
    a = at(x, env, R, C)
    b = at(y, env, R, C)
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        if op == "+":
            da, db = adj, adj
        elif op == "-":
            da, db = adj, -adj
        elif op in ("%", "*"):
            da, db = adj * b, adj * a
        elif op == "/":
            da, db = adj / b, -adj * a / (b * b)
        else:
            raise ValueError(op)
    _backprop(x, env, R, C, da, out)
    _backprop(y, env, R, C, db, out)


def local_adjoints(node, env, R, C, gL=1.0):
    """Reverse pass of an element-wise tree at output positions ``(R, C)``.

    Returns ``[(leaf name, leaf rows, leaf cols, adjoint), ...]``, one entry
    per leaf occurrence, with index arrays that broadcast to the adjoint's
    shape.
    """
    out = []
    shape = np.broadcast_shapes(np.shape(R), np.shape(C))
    _backprop(parse(node), env, R, C, np.full(shape, float(gL)), out)
    return out


def _scatter(env, occurrences):
    """Sum the occurrences' adjoints per stored element of each leaf.
    Returns ``{name: (flat indices, values)}``."""
    per_leaf = {}
    for name, Rl, Cl, adj in occurrences:
        buf = env[name]
        adj = np.asarray(adj, dtype=np.float64)
        Rb, Cb = np.broadcast_arrays(np.asarray(Rl, dtype=np.int64),
                                     np.asarray(Cl, dtype=np.int64))
        Rb = np.broadcast_to(Rb, adj.shape)
        Cb = np.broadcast_to(Cb, adj.shape)
        idx = (Rb + Cb * buf.ld).ravel()
        per_leaf.setdefault(name, []).append((idx, adj.ravel()))
    out = {}
    for name, parts in per_leaf.items():
        idx = np.concatenate([p[0] for p in parts])
        val = np.concatenate([p[1] for p in parts])
        uniq, inv = np.unique(idx, return_inverse=True)
        out[name] = (uniq, np.bincount(inv, weights=val, minlength=len(uniq)))
    return out


def _check_root(node):
    n = parse(node)
    if n.op != "accu":
        raise ValueError("the fused gradient is defined for accu(...) roots")
    return n.args[0]


def gradient(node, env, gL=1.0) -> dict:
    """Full gradient ``{leaf name: FP64 matrix of the leaf's shape}`` of
    ``gL * accu(f)``. Every output element is visited (small inputs)."""
    inner = _check_root(node)
    r, c = shape_of(inner, env)
    occ = local_adjoints(inner, env, np.arange(r)[:, None], np.arange(c)[None, :], gL)
    out = {}
    for name, (idx, val) in _scatter(env, occ).items():
        buf = env[name]
        flat = np.zeros(buf.ld * buf.cols)
        flat[idx] = val
        out[name] = flat.reshape(buf.cols, buf.ld).T[: buf.rows, :].copy()
    for name in env:
        if name not in out:
            b = env[name]
            out[name] = np.zeros((b.rows, b.cols))
    return out


def gradient_rows(node, env, rows, gL=1.0) -> dict:
    """Contribution of the output rows ``rows`` (all columns) to the gradient:
    ``{leaf name: (flat indices, values)}``.

    For a leaf read element for element (no ``t``) or as ``each_col``, the
    stored elements in those rows are read only by those output rows, so
    their entries here are the exact full gradient.
    """
    inner = _check_root(node)
    _, c = shape_of(inner, env)
    R = np.asarray(rows, dtype=np.int64)[:, None]
    occ = local_adjoints(inner, env, R, np.arange(c)[None, :], gL)
    return _scatter(env, occ)


# ---------------------------------------------------------------- error bound of a gradient
#
# sigma for the reverse pass, in units of the unit roundoff (first order):
# the adjoint handed to an operand is c = adj * p, where p is the node's
# local partial derivative computed from forward values; its bound is
#     sigma_c = sigma_adj |p| + |adj| sigma_p + |c|
# with sigma_p the bound of computing p from operands (value, sigma) as
# given by expr.at_sigma. Contributions summed into one stored element add
# the rounding of that sum (sum |c|). The root adjoint gL is exact.

def _partials_sigma(op, n, env, R, C):
    """[(operand node, p, sigma_p), ...] for one operator node."""
    from .expr import at_sigma, _apply_unary, _EXACT_UNARY
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        if op in UNARY:
            a, sa = at_sigma(n.args[0], env, R, C)
            z, sz = at_sigma(n, env, R, C)
            if op == "neg":
                return [(n.args[0], -np.ones_like(a), 0.0)]
            if op == "abs":
                return [(n.args[0], np.sign(a), 0.0)]
            if op == "exp":
                return [(n.args[0], z, sz)]
            if op == "log":
                p = 1.0 / a
                return [(n.args[0], p, sa / (a * a) + np.abs(p))]
            if op == "sqrt":
                p = 0.5 / z
                return [(n.args[0], p, 0.5 * sz / (z * z) + np.abs(p))]
            if op == "square":
                return [(n.args[0], 2.0 * a, 2.0 * sa)]
            if op == "sigmoid":
                p = z * (1.0 - z)
                return [(n.args[0], p, np.abs(1.0 - 2.0 * z) * sz + 2.0 * np.abs(p))]
            if op == "tanh":
                p = 1.0 - z * z
                return [(n.args[0], p, 2.0 * np.abs(z) * sz + z * z + np.abs(p))]
        if op == "pow":
            a, sa = at_sigma(n.args[0], env, R, C)
            k = n.args[1].value
            p = k * np.power(a, k - 1)
            return [(n.args[0], p, np.abs(k * (k - 1) * np.power(a, k - 2)) * sa + np.abs(p))]
        if op == "gt":
            return []
        x, y = n.args
        a, sa = at_sigma(x, env, R, C)
        b, sb = at_sigma(y, env, R, C)
        if op == "+":
            return [(x, 1.0, 0.0), (y, 1.0, 0.0)]
        if op == "-":
            return [(x, 1.0, 0.0), (y, -1.0, 0.0)]
        if op in ("%", "*"):
            return [(x, b, sb), (y, a, sa)]
        if op == "/":
            pa = 1.0 / b
            pb = -a / (b * b)
            spa = sb / (b * b) + np.abs(pa)
            spb = sa / (b * b) + 2.0 * np.abs(a) * sb / np.abs(b) ** 3 + 2.0 * np.abs(pb)
            return [(x, pa, spa), (y, pb, spb)]
    raise ValueError(op)


def _backprop_sigma(n, env, R, C, adj, sadj, out):
    op = n.op
    if op == "num":
        return
    if op == "leaf":
        out.append((n.name, R, C, adj, sadj))
        return
    if op == "t":
        _backprop_sigma(n.args[0], env, C, R, adj, sadj, out)
        return
    if op == "each_col":
        _backprop_sigma(n.args[0], env, R, np.zeros_like(np.asarray(C)), adj, sadj, out)
        return
    if op == "each_row":
        _backprop_sigma(n.args[0], env, np.zeros_like(np.asarray(R)), C, adj, sadj, out)
        return
    if _is_product(n):
        raise ValueError("no fused gradient through a matrix product")
    for child, p, sp in _partials_sigma(op, n, env, R, C):
        if child.op == "num":
            continue
        with np.errstate(over="ignore", invalid="ignore"):
            c = adj * p
            sc = sadj * np.abs(p) + np.abs(adj) * sp + np.abs(c)
        _backprop_sigma(child, env, R, C, c, sc, out)


def gradient_sigma(node, env, gL=1.0, rows=None) -> dict:
    """``{leaf name: (flat indices, gradient values, sigma)}`` of ``gL * accu(f)``
    over every output element, or over the output rows ``rows`` (see
    ``gradient_rows`` for when that gives exact entries)."""
    inner = _check_root(node)
    r, c = shape_of(inner, env)
    R = np.arange(r)[:, None] if rows is None else np.asarray(rows, dtype=np.int64)[:, None]
    Cc = np.arange(c)[None, :]
    shape = np.broadcast_shapes(R.shape, Cc.shape)
    occ = []
    _backprop_sigma(parse(inner), env, R, Cc, np.full(shape, float(gL)), np.zeros(shape), occ)
    vals = _scatter(env, [(nm, Rl, Cl, a) for nm, Rl, Cl, a, _ in occ])
    sigs = _scatter(env, [(nm, Rl, Cl, s + np.abs(a)) for nm, Rl, Cl, a, s in occ])
    out = {}
    for name, (idx, v) in vals.items():
        idx2, s = sigs[name]
        assert np.array_equal(idx, idx2)
        out[name] = (idx, v, s)
    return out
