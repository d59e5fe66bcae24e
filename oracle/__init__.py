"""FP64 CPU oracle for fused expression evaluation (TEST INFRASTRUCTURE ONLY).

This package is the checker, not the product. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it. It shares no code with the CUDA library and never imports it;
both sides take their inputs from ``synth``.

What it computes (Curtin, Edel, Sanderson, "Fast GPU Linear Algebra via
Compile Time Expression Fusion"):

* Sec. 3: an expression is a tree; element ``(row, col)`` of a leaf matrix is
  ``in[row + col*n_rows]`` (with a leading dimension, ``in[row + col*ld]``),
  a transpose swaps ``row`` and ``col`` before the inner access, and a scalar
  node wraps the inner access (``... + aux``). ``expr.at`` is that rule,
  vectorised over arrays of indices.
* Sec. 4: the operators of the expression suite (``+ - % /``, scalar scale,
  ``exp log sqrt abs square pow tanh``, sigmoid ``1/(1+exp(-x))``, the mask
  ``X > 0``, ``.t()``) and the reductions named in Sec. 3 (``accu``), plus
  ``sum``/``max`` along a dimension and the 2-norm.
* Reductions use Neumaier-compensated FP64 summation (``sums.py``).
* ``grad.py``: reverse-mode derivative of ``accu(f(leaves))``.
* ``compare.py``: the scaled error of a computed result against the oracle's
  value, scaled by its error bound ``at_sigma`` or magnitude ``at_mag``.

Every value is FP64; inputs are the exact FP64 values of the stored
(rounded) elements. Sums are the plain mathematical definitions; the only
freedom is rounding order, which compensated summation makes negligible.
"""
from .expr import (Node, parse, shape_of, leaves_of, at, at_sigma, at_mag, evaluate,
                   evaluate_sigma, evaluate_mag, REDUCTIONS)
from .sums import neumaier, neumaier_axis
from .grad import local_adjoints, gradient, gradient_rows

__all__ = ["Node", "parse", "shape_of", "leaves_of", "at", "at_sigma", "at_mag", "evaluate",
           "evaluate_sigma", "evaluate_mag", "REDUCTIONS", "neumaier", "neumaier_axis", "local_adjoints",
           "gradient", "gradient_rows"]
