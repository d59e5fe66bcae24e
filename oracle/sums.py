"""Neumaier-compensated FP64 summation (oracle; test infrastructure only).

Neumaier's improvement of Kahan summation (A. Neumaier, 1974): keep a
running sum ``s`` and a correction ``c``; for each term ``x``,
``t = s + x``; the rounding error of that addition is ``(s - t) + x`` when
``|s| >= |x|`` and ``(x - t) + s`` otherwise; add it to ``c``; ``s = t``.
The result is ``s + c``. Its error is about ``2u|sum|`` plus a term of order
``n u^2 sum|x|``, so summing 2.7e8 terms stays far inside a 1e-13 bound,
which a plain sequential FP64 sum (error up to ``n u sum|x|``) would not.
"""
from __future__ import annotations

import numpy as np


def neumaier(values) -> float:
    """Compensated sum of a 1-D sequence, in order."""
    s = 0.0
    c = 0.0
    for x in np.asarray(values, dtype=np.float64).ravel().tolist():
        t = s + x
        if abs(s) >= abs(x):
            c += (s - t) + x
        else:
            c += (x - t) + s
        s = t
    return s + c


def neumaier_axis(a: np.ndarray, axis: int, state=None):
    """Compensated sums along ``axis``, vectorised across the other axis.

    Steps through the slices of ``axis`` in order, each slice updating one
    Neumaier accumulator per position of the other axis. ``state`` carries
    ``(s, c)`` from an earlier call so that a sum can run over panels;
    returns the new ``(s, c)``; the sums are ``s + c``.
    """
    a = np.asarray(a, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("neumaier_axis expects a 2-D array")
    n_other = a.shape[1 - axis]
    if state is None:
        s = np.zeros(n_other)
        c = np.zeros(n_other)
    else:
        s, c = state
        s = s.copy()
        c = c.copy()
    for k in range(a.shape[axis]):
        x = a[k, :] if axis == 0 else a[:, k]
        t = s + x
        big = np.abs(s) >= np.abs(x)
        with np.errstate(invalid="ignore"):
            err = np.where(big, (s - t) + x, (x - t) + s)
        # once a sum has overflowed, its correction carries no information
        c += np.where(np.isfinite(t), err, 0.0)
        s = t
    return s, c
