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
