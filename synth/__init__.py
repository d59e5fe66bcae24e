"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module draws random matrices and rounds them to a storage type. It
holds none of the expression arithmetic: the oracle (under ``oracle/``) and
the CUDA library (``paper_2604_22242_gb300``) both consume the buffers made
here, and neither imports the other.

Recipe (the same on every machine):

* ``numpy.random.Generator(PCG64(...))``; one child stream per operand from
  ``SeedSequence(seed).spawn(k)``, in the order the operands are listed.
* Values are drawn in FP64, in column-major element order (element ``(r, c)``
  is draw number ``r + c*rows``), then rounded once, to nearest with ties to
  even, to the storage type.
* Buffers are flat and column-major with leading dimension ``ld`` (the
  storage convention of the paper's Sec. 3 element-access rule,
  ``in[row + col*n_rows]``).

Storage types: ``f32``, ``f64``, ``f16`` (numpy float16) and ``bf16``
(kept as ``uint16`` bit patterns, since numpy has no bfloat16).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

STORAGES = ("f32", "f64", "bf16", "f16")

_NP_STORAGE = {"f32": np.float32, "f64": np.float64, "f16": np.float16, "bf16": np.uint16}

# (significand bits incl. the implicit one, smallest subnormal exponent, largest finite)
_FORMAT = {
    "bf16": (8, -133, float.fromhex("0x1.fep127")),
    "f16": (11, -24, 65504.0),
}


def storage_nbytes(storage: str) -> int:
    return {"f32": 4, "f64": 8, "bf16": 2, "f16": 2}[storage]


def _round_small_format(x: np.ndarray, storage: str) -> np.ndarray:
    """Round FP64 values once, to nearest-even, onto the bf16/f16 grid.

    The spacing of representable numbers around ``x`` is
    ``2**(e - p)`` for ``x = m * 2**e`` with ``0.5 <= |m| < 1`` and ``p``
    significand bits, floored at the subnormal spacing. ``np.rint`` rounds
    half to even. Values past the largest finite number go to +-inf, as IEEE
    round-to-nearest does once they reach the midpoint to the next binade.
    """
    p, qmin, fmax = _FORMAT[storage]
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    q = np.maximum(e - p, qmin).astype(np.float64)
    y = np.rint(np.ldexp(x, -q.astype(np.int64))) * np.exp2(q)
    # IEEE overflow threshold: fmax + half an ulp of fmax rounds to inf.
    ulp_max = math.ldexp(1.0, math.frexp(fmax)[1] - p)
    over = np.abs(x) >= fmax + 0.5 * ulp_max
    y = np.where(over, np.copysign(np.inf, x), y)
    y = np.where(np.isnan(x), np.nan, y)
    return y


def round_to_storage(x64: np.ndarray, storage: str) -> np.ndarray:
    """FP64 -> storage array (single round-to-nearest-even)."""
    x64 = np.asarray(x64, dtype=np.float64)
    if storage == "f64":
        return x64.copy()
    if storage == "f32":
        return x64.astype(np.float32)
    if storage == "f16":
        return _round_small_format(x64, "f16").astype(np.float16)
    if storage == "bf16":
        y = _round_small_format(x64, "bf16").astype(np.float32)  # exact: 8 significand bits
        return (y.view(np.uint32) >> np.uint32(16)).astype(np.uint16)
    raise ValueError(f"unknown storage {storage!r}")


def to_f64(buf: np.ndarray, storage: str) -> np.ndarray:
    """Exact FP64 value of every stored element (a format decode, no rounding)."""
    buf = np.asarray(buf)
    if storage == "bf16":
        return (buf.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    return buf.astype(np.float64)


def draw(rng: np.random.Generator, n: int, dist: str) -> np.ndarray:
    """``n`` FP64 draws of one distribution from one stream."""
    if dist == "uniform":          # i.i.d. U[-1, 1]
        return rng.uniform(-1.0, 1.0, n)
    if dist == "normal":           # N(0, 1)
        return rng.normal(0.0, 1.0, n)
    if dist == "normal_half":      # N(0, sd 0.5)
        return rng.normal(0.0, 0.5, n)
    if dist == "lognormal_signed": # lognormal(0, 1) times a fair random sign
        mag = rng.lognormal(0.0, 1.0, n)
        sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
        return mag * sign
    if dist == "positive":         # U[0.5, 2], for trees that need x > 0 (log)
        return rng.uniform(0.5, 2.0, n)
    raise ValueError(f"unknown distribution {dist!r}")


@dataclasses.dataclass
class Buffer:
    """A column-major matrix in storage form: element (r, c) is ``data[r + c*ld]``."""
    data: np.ndarray
    rows: int
    cols: int
    ld: int
    storage: str

    def f64(self) -> np.ndarray:
        return to_f64(self.data, self.storage)


def matrix(rng: np.random.Generator, rows: int, cols: int, dist: str, storage: str,
           ld: int | None = None, fill: float = 0.0) -> Buffer:
    """One matrix; padding rows (``ld > rows``) hold ``fill`` and are never drawn."""
    ld = max(rows, 1) if ld is None else ld
    if ld < max(rows, 1):
        raise ValueError("ld must be >= rows")
    vals = draw(rng, rows * cols, dist)
    if ld == rows:
        flat = vals
    else:
        flat = np.full(ld * cols, fill, dtype=np.float64)
        flat.reshape(cols, ld)[:, :rows] = vals.reshape(cols, rows)
    return Buffer(round_to_storage(flat, storage), rows, cols, ld, storage)


def operands(seed: int, specs, storage: str, dist: str, lds: dict | None = None) -> dict:
    """Matrices for named operands, one child stream each, in ``specs`` order.

    ``specs`` is a list of ``(name, rows, cols)``; ``lds`` optionally maps a
    name to a leading dimension larger than its row count. Large operands
    are drawn on a thread pool, one operand per thread: every operand has
    its own stream, so the values do not depend on the threading.
    """
    lds = lds or {}
    kids = np.random.SeedSequence(seed).spawn(len(specs))

    def one(job):
        (name, r, c), ss = job
        return name, matrix(np.random.Generator(np.random.PCG64(ss)), r, c, dist, storage,
                            ld=lds.get(name))

    jobs = list(zip(specs, kids))
    big = sum(r * c for _, r, c in specs) >= (1 << 22) and len(specs) > 1
    if big:
        import concurrent.futures as cf
        import os
        with cf.ThreadPoolExecutor(min(len(jobs), os.cpu_count() or 1)) as ex:
            return dict(ex.map(one, jobs))
    return dict(one(j) for j in jobs)


def batch_shapes(seed: int, count: int, lo: int = 16, hi: int = 2048):
    """Rows and cols of a batch, each log-uniform in [lo, hi].

    Drawn from child 0 of ``SeedSequence(seed)``: rows then cols for matrix 0,
    then matrix 1, and so on; ``round(exp(U(ln lo, ln hi)))``.
    """
    ss = np.random.SeedSequence(seed).spawn(1)[0]
    rng = np.random.Generator(np.random.PCG64(ss))
    u = rng.uniform(math.log(lo), math.log(hi), 2 * count)
    rc = np.rint(np.exp(u)).astype(np.int64)
    return rc[0::2].copy(), rc[1::2].copy()


def batch_operands(seed: int, count: int, layout, storage: str = "f32", dist: str = "uniform",
                   lo: int = 16, hi: int = 2048, count_max: int | None = None):
    """Per-matrix operands of a batch.

    ``layout`` lists ``(name, transposed)``: a transposed operand of matrix
    ``i`` is ``cols_i x rows_i``. Operand ``k`` draws from child ``k + 1`` of
    ``SeedSequence(seed)`` (child 0 drew the shapes), matrix after matrix.
    Returns ``(rows, cols, {name: [Buffer, ...]})``.
    """
    rows, cols = batch_shapes(seed, count, lo, hi)
    kids = np.random.SeedSequence(seed).spawn(len(layout) + 1)[1:]

    def one(job):
        (name, tr), ss = job
        rng = np.random.Generator(np.random.PCG64(ss))
        mats = []
        for r, c in zip(rows.tolist(), cols.tolist()):
            rr, cc = (c, r) if tr else (r, c)
            mats.append(matrix(rng, rr, cc, dist, storage))
        return name, mats

    # one operand per thread (each has its own stream: same values either way)
    import concurrent.futures as cf
    import os
    with cf.ThreadPoolExecutor(max(1, min(len(layout), os.cpu_count() or 1))) as ex:
        out = dict(ex.map(one, list(zip(layout, kids))))
    return rows, cols, out
