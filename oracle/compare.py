"""Scaled error of a computed result against the oracle (test infrastructure only).

The oracle gives, per output element, its FP64 value ``z`` and two scales:
``sigma`` (``expr.at_sigma``, a first-order running error bound that
follows errors through transcendental arguments) and ``m``
(``expr.at_mag``, the magnitude scale of the tree evaluated on absolute
values). A computed element ``g`` is judged by

    err = |g - z| / max(scale, |z|, tiny)

with ``scale = m`` for trees built only from + - % scalar ops, neg, abs,
square, the mask gt, transposes, broadcasts and sums/maxima/norms over
them, where rounding errors are bounded by a small multiple of ``u m``
(Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1-3.3 and
4.2), and ``scale = sigma`` for trees with exp, log, sqrt, sigmoid, tanh,
pow, a division or a matrix product, where an error in an argument is
amplified by a derivative that ``m`` does not see.

Outputs whose oracle value exceeds the storage type's largest finite value
must come out as an infinity of the oracle's sign (or that largest finite
value, at the rounding edge); they are counted and left out of the maximum.
FP16 outputs below the normal range pass within one subnormal step (2^-24)
of the oracle, and beyond that only when the gap is within tolerance of the
scale (cancellation).
"""
from __future__ import annotations

import numpy as np

from .expr import parse

MAXFIN = {"f32": float(np.finfo(np.float32).max), "f64": float(np.finfo(np.float64).max),
          "bf16": float.fromhex("0x1.fep127"), "f16": 65504.0}
TINY = {"f32": 2.0**-126, "f64": 2.0**-1022, "bf16": 2.0**-126, "f16": 2.0**-14}

# operators whose rounding errors the magnitude scale does not bound
_NEEDS_SIGMA = {"exp", "log", "sqrt", "sigmoid", "tanh", "pow", "/"}
_TRANSCENDENTAL = {"exp", "log", "sqrt", "sigmoid", "tanh", "pow"}

# Tolerances on the scaled error, by storage type: element-wise results,
# element-wise results through transcendental functions, and reductions
# (every reduction of an FP32, BF16 or FP16 tree comes out in FP32 from a
# compensated FP32 accumulation, so all of them are held to the FP32
# reduction bound).
TOL_EW = {"f64": 1e-13, "f32": 2e-6, "bf16": 8e-3, "f16": 1e-3}
TOL_TRANS = {"f64": 1e-13, "f32": 1e-5, "bf16": 8e-3, "f16": 1e-3}
TOL_RED = {"f64": 1e-13, "f32": 1e-5, "bf16": 1e-5, "f16": 1e-5}


def _has(tree, ops) -> bool:
    def rec(x):
        return x.op in ops or any(rec(a) for a in x.args)
    return rec(parse(tree))


def tolerance(tree, storage, reduction=False) -> float:
    """The bound a result of `tree` with `storage` is held to: the reduction
    bound for a reduced output (accu, norm, sum or max along a dimension,
    or a gradient of one), the transcendental bound when the tree has exp,
    log, sqrt, sigmoid, tanh or pow, the element-wise bound otherwise."""
    root = parse(tree)
    if reduction or root.op in ("accu", "norm", "sum", "max"):
        return TOL_RED[storage]
    return TOL_TRANS[storage] if _has(tree, _TRANSCENDENTAL) else TOL_EW[storage]


def gate_scale(tree) -> str:
    """``"m"`` or ``"sigma"``: the scale a tree's results are judged by."""
    n = parse(tree)

    def rec(x):
        if x.op in _NEEDS_SIGMA:
            return True
        if x.op == "*" and x.args[0].op != "num" and x.args[1].op != "num":
            return True        # a matrix product: a K-term dot product per element
        return any(rec(a) for a in x.args)

    return "sigma" if rec(n) else "m"


def scaled_error(gpu, ref, scale, storage):
    """(max scaled error, #expected overflows, #bad non-finite, max plain rel)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.broadcast_to(np.asarray(scale, dtype=np.float64), ref.shape)
    over = np.abs(ref) > MAXFIN[storage]
    bad = 0
    if np.any(over):
        okinf = np.isinf(gpu[over]) & (np.sign(gpu[over]) == np.sign(ref[over]))
        okmax = np.abs(gpu[over]) == MAXFIN[storage]
        bad += int(np.sum(~(okinf | okmax)))
    fin = ~over
    g, r, s = gpu[fin], ref[fin], scale[fin]
    bad += int(np.sum(~np.isfinite(g)))
    g = np.where(np.isfinite(g), g, np.inf)
    denom = np.maximum(np.maximum(s, np.abs(r)), TINY[storage])
    err = np.abs(g - r) / denom
    if storage == "f16":
        sub = np.abs(r) < 2.0**-14
        d = np.abs(g[sub] - r[sub])
        with np.errstate(divide="ignore", invalid="ignore"):
            esub = np.where(d <= 2.0**-24, 0.0, d / np.maximum(s[sub], np.abs(r[sub])))
        err[sub] = np.nan_to_num(esub, nan=np.inf)
    nz = np.abs(r) > TINY[storage]
    rel = float(np.max(np.abs(g[nz] - r[nz]) / np.abs(r[nz]))) if np.any(nz) else 0.0
    return (float(np.max(err)) if err.size else 0.0), int(np.sum(over)), bad, rel


def _nanmax(a, b):
    if a != a:
        return b
    if b != b:
        return a
    return max(a, b)


class ErrorReport:
    """Running summary of a result compared piece by piece (column panels,
    sampled positions, matrices of a batch): the maxima of the scaled error
    under sigma and under m, of the plain relative error, and the counts of
    wrong non-finite outputs and of expected overflows."""

    def __init__(self, storage, tol, gate):
        self.storage, self.tol, self.gate = storage, tol, gate
        self.err_sigma = self.err_mag = float("nan")   # nan: that scale was not computed
        self.rel = 0.0
        self.nonfinite = self.overflow = 0
        self.n = 0

    def add(self, gpu, ref, sigma=None, mag=None):
        """Compares one piece; the gate's scale must be given, the other is
        optional (reported only)."""
        first, other = (mag, sigma) if self.gate == "m" else (sigma, mag)
        if first is None:
            raise ValueError(f"the {self.gate} scale is needed to gate this result")
        e, over, bad, rel = scaled_error(gpu, ref, first, self.storage)
        e2 = scaled_error(gpu, ref, other, self.storage)[0] if other is not None else float("nan")
        es, em = (e2, e) if self.gate == "m" else (e, e2)
        self.err_sigma = _nanmax(self.err_sigma, es)
        self.err_mag = _nanmax(self.err_mag, em)
        self.rel = max(self.rel, rel)
        self.nonfinite += bad
        self.overflow += over
        self.n += int(np.size(ref))
        return self

    def merge(self, other):
        """Fold another report of the same output into this one."""
        self.err_sigma = _nanmax(self.err_sigma, other.err_sigma)
        self.err_mag = _nanmax(self.err_mag, other.err_mag)
        self.rel = max(self.rel, other.rel)
        self.nonfinite += other.nonfinite
        self.overflow += other.overflow
        self.n += other.n
        return self

    @property
    def err(self):
        """The gated error (the one held to the tolerance)."""
        return self.err_mag if self.gate == "m" else self.err_sigma

    @property
    def ok(self):
        return self.nonfinite == 0 and self.err <= self.tol

    def as_dict(self):
        def num(x):
            return None if x != x else float(x)
        return {"max_scaled_err_sigma": num(self.err_sigma),
                "max_scaled_err_m": num(self.err_mag), "max_plain_rel_err": float(self.rel),
                "tol": self.tol, "gate": self.gate, "nonfinite": self.nonfinite,
                "overflow_expected": self.overflow, "compared": self.n}
