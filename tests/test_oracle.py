"""Pins for the FP64 oracle: worked examples, closed forms, brute force,
library routines and finite differences. CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import expr as oexpr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def buf(values_colmajor, rows, cols, ld=None, storage="f64"):
    ld = rows if ld is None else ld
    flat = np.zeros(ld * cols)
    v = np.asarray(values_colmajor, dtype=np.float64).reshape(cols, rows)
    flat.reshape(cols, ld)[:, :rows] = v
    return synth.Buffer(synth.round_to_storage(flat, storage), rows, cols, ld, storage)


def rand_env(seed, specs, dist="uniform", storage="f64"):
    return synth.operands(seed, specs, storage, dist)


# ------------------------------------------------------------ Sec. 3 worked example

def _read_golden(name):
    fields = {}
    expect = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "expect":
                expect.append([float(v) for v in vals])
            else:
                fields[key] = [float(v) for v in vals]
    return fields, np.array(expect)


def test_worked_example_trans_plus_scalar():
    f, expect = _read_golden("worked_example_trans_plus_scalar.txt")
    r, c = int(f["rows"][0]), int(f["cols"][0])
    X = buf(f["data"], r, c)
    env = {"X": X}
    got = oracle.evaluate(f"(+ (t X) {f['aux'][0]})", env)
    assert got.shape == (int(f["expect_rows"][0]), int(f["expect_cols"][0]))
    assert np.array_equal(got, expect)
    # and the printed access rule, index by index: in[col + row*n_rows] + aux
    for row in range(c):
        for col in range(r):
            assert got[row, col] == X.data[col + row * r] + f["aux"][0]


def test_hand_values():
    with open(os.path.join(GOLDEN, "hand_values.txt")) as fh:
        lines = [l.strip() for l in fh if l.strip() and not l.startswith("#")]
    assert len(lines) >= 8
    for line in lines:
        name, rest = line.split(" ", 1)
        ex_end = rest.rindex(")") + 1
        ex = rest[:ex_end]
        leaves, shape, expected = rest[ex_end:].split()
        r, c = (int(x) for x in shape.split("x"))
        env = {}
        for part in leaves.split(";"):
            k, v = part.split("=")
            vals = [float(x) for x in v.split(",")]
            env[k] = buf(vals, r, c) if len(vals) == r * c else buf(vals, len(vals), 1)
        got = oracle.evaluate(ex, env)
        want = np.array([float(x) for x in expected.split(",")])
        assert np.allclose(got.T.ravel(), want, rtol=0, atol=1e-15), name


# ------------------------------------------------------------ layout and transpose

def test_leaf_layout_with_leading_dimension():
    rows, cols, ld = 3, 4, 5
    vals = np.arange(rows * cols, dtype=np.float64) * 1.5 - 4
    X = buf(vals, rows, cols, ld=ld)
    got = oracle.evaluate("(abs X)", {"X": X})
    for r in range(rows):
        for c in range(cols):
            assert got[r, c] == abs(X.data[r + c * ld])


def test_trans_trans_is_identity_and_swaps():
    env = rand_env(5, [("X", 7, 4)])
    X = oracle.evaluate("(+ X 0)", env)
    assert np.array_equal(oracle.evaluate("(t (t X))", env), X)
    assert np.array_equal(oracle.evaluate("(t X)", env), X.T)


def test_exact_identities():
    env = rand_env(6, [("X", 9, 8), ("Y", 9, 8)], "normal")
    assert np.all(oracle.evaluate("(- X X)", env) == 0.0)
    assert np.array_equal(oracle.evaluate("(square X)", env), oracle.evaluate("(% X X)", env))
    assert np.array_equal(oracle.evaluate("(neg (neg X))", env), oracle.evaluate("(+ X 0)", env))
    assert np.array_equal(oracle.evaluate("(* 2 X)", env), oracle.evaluate("(+ X X)", env))


def test_transcendental_identities():
    env = rand_env(7, [("X", 10, 10)], "positive")
    x = oracle.evaluate("(+ X 0)", env)
    assert np.max(np.abs(oracle.evaluate("(exp (log X))", env) - x) / x) < 4e-16
    envn = rand_env(8, [("X", 10, 10)], "normal")
    xn = oracle.evaluate("(+ X 0)", envn)
    s = oracle.evaluate("(sqrt (abs X))", envn)
    assert np.max(np.abs(s * s - np.abs(xn)) / np.abs(xn)) < 4e-16
    sg = oracle.evaluate("(sigmoid X)", envn)
    sgn = oracle.evaluate("(sigmoid (neg X))", envn)
    assert np.max(np.abs(sg + sgn - 1.0)) < 4e-16
    scipy_special = pytest.importorskip("scipy.special")
    assert np.max(np.abs(sg - scipy_special.expit(xn))) < 4e-16
    th = oracle.evaluate("(tanh X)", envn)
    assert np.max(np.abs(th - (2 * scipy_special.expit(2 * xn) - 1))) < 1e-15
    p3 = oracle.evaluate("(pow X 3)", envn)
    assert np.max(np.abs(p3 - xn * xn * xn)) <= 4e-16 * np.max(np.abs(xn) ** 3)


# ------------------------------------------------------------ reductions: closed forms

def test_accu_of_ones():
    for r, c in [(1, 1), (3, 5), (64, 33), (1000, 7)]:
        env = {"X": buf(np.ones(r * c), r, c)}
        assert oracle.evaluate("(accu X)", env)[0, 0] == r * c


def test_accu_arithmetic_series():
    r, c = 300, 211
    n = r * c
    env = {"X": buf(np.arange(n, dtype=np.float64), r, c)}   # X(r, c) = r + c*rows
    assert oracle.evaluate("(accu X)", env)[0, 0] == n * (n - 1) / 2


def test_dim_reductions_closed_forms():
    r, c = 37, 23
    colidx = np.repeat(np.arange(c, dtype=np.float64), r)      # X(r, c) = c
    rowidx = np.tile(np.arange(r, dtype=np.float64), c)        # X(r, c) = r
    env = {"X": buf(colidx, r, c), "Y": buf(rowidx, r, c)}
    assert np.array_equal(oracle.evaluate("(sum X 0)", env)[0], np.arange(c) * r)
    assert np.array_equal(oracle.evaluate("(max X 1)", env)[:, 0], np.full(r, c - 1.0))
    assert np.array_equal(oracle.evaluate("(sum X 1)", env)[:, 0], np.full(r, c * (c - 1) / 2))
    assert np.array_equal(oracle.evaluate("(max Y 0)", env)[0], np.full(c, r - 1.0))
    assert np.array_equal(oracle.evaluate("(sum Y 1)", env)[:, 0], np.arange(r) * c)


def test_norm_closed_forms():
    r, c = 50, 40
    env = {"X": buf(np.ones(r * c), r, c)}
    assert oracle.evaluate("(norm X)", env)[0, 0] == math.sqrt(r * c)
    env = rand_env(9, [("X", 31, 17), ("Y", 31, 17)], "normal")
    a = oracle.evaluate("(norm (- X Y))", env)[0, 0]
    b = math.sqrt(oracle.evaluate("(accu (square (- X Y)))", env)[0, 0])
    assert abs(a - b) <= 2e-16 * a
    d = env["X"].f64() - env["Y"].f64()
    assert abs(a - np.linalg.norm(d)) <= 1e-15 * a


def test_reductions_nan_propagates_in_max():
    X = buf([1.0, np.nan, 3.0, 4.0], 2, 2)
    m1 = oracle.evaluate("(max X 1)", {"X": X})
    m0 = oracle.evaluate("(max X 0)", {"X": X})
    assert np.isnan(m1[1, 0]) and m1[0, 0] == 3.0
    assert np.isnan(m0[0, 0]) and m0[0, 1] == 4.0


# ------------------------------------------------------------ compensated sums

def test_neumaier_beats_cancellation():
    assert oracle.neumaier([1e16, 1.0, -1e16]) == 1.0
    s, c = oracle.neumaier_axis(np.array([[1e16, 1.0, -1e16]]), axis=1)
    assert s[0] + c[0] == 1.0
    s, c = oracle.neumaier_axis(np.array([[1e16], [1.0], [-1e16]]), axis=0)
    assert s[0] + c[0] == 1.0


def test_neumaier_matches_fsum():
    rng = np.random.default_rng(11)
    for scale in (1.0, 1e8):
        x = rng.normal(size=200_000) * scale
        ref = math.fsum(x)
        s, c = oracle.neumaier_axis(x.reshape(400, 500), axis=0)
        got = oracle.neumaier(np.stack([s, c], 1).ravel())
        assert abs(got - ref) <= 2 * math.ulp(ref) + 1e-300
        assert abs(oracle.neumaier(x[:20000]) - math.fsum(x[:20000])) <= 2 * math.ulp(ref)


def test_long_sum_of_float32_tenths():
    # 2^22 copies of fl32(0.1): the exact sum n*fl32(0.1) is representable in FP64
    n = 1 << 22
    x = float(np.float32(0.1))
    rows, cols = 2048, 2048
    env = {"X": synth.Buffer(np.full(n, np.float32(0.1)), rows, cols, rows, "f32")}
    assert oracle.evaluate("(accu X)", env)[0, 0] == n * x


def test_integer_sums_exact():
    rng = np.random.default_rng(12)
    v = rng.integers(-1000, 1000, size=600 * 300).astype(np.float64)
    env = {"X": buf(v, 600, 300)}
    assert oracle.evaluate("(accu X)", env)[0, 0] == float(np.sum(v.astype(np.int64)))
    cs = oracle.evaluate("(sum X 0)", env)[0]
    assert np.array_equal(cs, v.reshape(300, 600).astype(np.int64).sum(1).astype(np.float64))


# ------------------------------------------------------------ brute force on tiny shapes

SHAPES = [(1, 1), (1, 6), (6, 1), (3, 5), (7, 7)]


def _el(b, r, c):
    return float(synth.to_f64(b.data[r + c * b.ld : r + c * b.ld + 1], b.storage)[0])


@pytest.mark.parametrize("rc", SHAPES)
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
def test_brute_force_schur_exp_trans(rc, storage):
    r, c = rc
    env = synth.operands(0, [("A", r, c), ("B", r, c), ("C", r, c), ("D", c, r)], storage,
                         "uniform")
    got = oracle.evaluate("(- (+ (% A B) (* 3.5 (exp C))) (t D))", env)
    for i in range(r):
        for j in range(c):
            want = (_el(env["A"], i, j) * _el(env["B"], i, j) + 3.5 * math.exp(_el(env["C"], i, j))
                    - _el(env["D"], j, i))
            assert got[i, j] == pytest.approx(want, rel=1e-15, abs=1e-15)


@pytest.mark.parametrize("rc", SHAPES)
def test_brute_force_schur_sqrt_sigmoid_and_reductions(rc):
    r, c = rc
    env = synth.operands(1, [("X", r, c), ("Y", r, c), ("W", r, c), ("V", r, c)], "f32",
                         "normal")
    Z = oracle.evaluate("(+ (% X Y) (/ (sqrt (abs W)) (+ 1 (exp (neg V)))))", env)
    cs = oracle.evaluate("(sum (% X Y) 0)", env)
    rm = oracle.evaluate("(max (abs (- X Y)) 1)", env)
    nr = oracle.evaluate("(norm (- X Y))", env)[0, 0]
    e = {k: (lambda b: (lambda i, j: _el(b, i, j)))(v) for k, v in env.items()}
    ssq = 0.0
    for j in range(c):
        col = 0.0
        for i in range(r):
            x, y, w, v = e["X"](i, j), e["Y"](i, j), e["W"](i, j), e["V"](i, j)
            want = x * y + math.sqrt(abs(w)) / (1.0 + math.exp(-v))
            assert Z[i, j] == pytest.approx(want, rel=1e-15, abs=1e-15)
            col += x * y
            ssq += (x - y) ** 2
        assert cs[0, j] == pytest.approx(col, rel=1e-14, abs=1e-14)
    for i in range(r):
        want = max(abs(e["X"](i, j) - e["Y"](i, j)) for j in range(c))
        assert rm[i, 0] == want
    assert nr == pytest.approx(math.sqrt(ssq), rel=1e-14)


@pytest.mark.parametrize("rc", SHAPES)
def test_brute_force_broadcast_sigmoid_loss(rc):
    r, c = rc
    env = synth.operands(3, [("X", r, c), ("W", r, c), ("Y", r, c), ("b", r, 1)], "f32",
                         "normal_half")
    L = oracle.evaluate("(accu (square (- (sigmoid (+ (% X W) (each_col b))) Y)))", env)[0, 0]
    want = 0.0
    for i in range(r):
        for j in range(c):
            u = _el(env["X"], i, j) * _el(env["W"], i, j) + _el(env["b"], i, 0)
            s = 1.0 / (1.0 + math.exp(-u))
            want += (s - _el(env["Y"], i, j)) ** 2
    assert L == pytest.approx(want, rel=1e-14)


def test_each_row_broadcast():
    env = synth.operands(4, [("X", 4, 6), ("b", 1, 6)], "f64", "normal")
    got = oracle.evaluate("(- X (each_row b))", env)
    for i in range(4):
        for j in range(6):
            assert got[i, j] == _el(env["X"], i, j) - _el(env["b"], 0, j)


def test_matrix_product_boundary():
    env = synth.operands(4, [("X", 5, 3), ("Y", 4, 3)], "f64", "normal")
    got = oracle.evaluate("(* 2 (* X (t Y)))", env)           # Fig. 1: Z = 2 X Y^T
    X = env["X"].f64().reshape(3, 5).T
    Y = env["Y"].f64().reshape(3, 4).T
    for i in range(5):
        for j in range(4):
            assert got[i, j] == pytest.approx(2 * sum(X[i, k] * Y[j, k] for k in range(3)),
                                              rel=1e-14)


def test_shape_errors():
    env = synth.operands(4, [("X", 4, 6), ("Y", 6, 4), ("b", 4, 1)], "f64", "normal")
    with pytest.raises(ValueError):
        oracle.evaluate("(+ X Y)", env)
    with pytest.raises(ValueError):
        oracle.evaluate("(+ Y (each_col b))", env)
    with pytest.raises(ValueError):
        oracle.parse("(exp X Y)")
    with pytest.raises(ValueError):
        oracle.parse("(frobnicate X)")


# ------------------------------------------------------------ error bound sigma

def _f32_eval(node, env, R, C):
    """Step-by-step FP32 evaluation (numpy float32 per operation); used only
    to check that sigma bounds a real rounding error."""
    n = oracle.parse(node)
    op = n.op
    f = np.float32
    if op == "num":
        return f(n.value)
    if op == "leaf":
        return oexpr._leaf_values(env[n.name], R, C).astype(f)
    if op == "t":
        return _f32_eval(n.args[0], env, C, R)
    if op == "each_col":
        return _f32_eval(n.args[0], env, R, np.zeros_like(C))
    a = _f32_eval(n.args[0], env, R, C)
    if op in oexpr.UNARY:
        return {"neg": lambda: -a, "exp": lambda: np.exp(a), "log": lambda: np.log(a),
                "sqrt": lambda: np.sqrt(a), "abs": lambda: np.abs(a),
                "square": lambda: a * a, "sigmoid": lambda: f(1) / (f(1) + np.exp(-a)),
                "tanh": lambda: np.tanh(a)}[op]().astype(f)
    b = _f32_eval(n.args[1], env, R, C)
    return {"+": lambda: a + b, "-": lambda: a - b, "%": lambda: a * b, "*": lambda: a * b,
            "/": lambda: a / b, "gt": lambda: a > b}[op]().astype(f)


TREES = [
    "(- (+ (% A B) (* 3.5 (exp C))) (t D))",
    "(+ (% A B) (/ (sqrt (abs C)) (+ 1 (exp (neg D)))))",
    "(- (sigmoid (+ (% A B) (each_col b))) C)",
    "(+ (- A B) (- C (t D)))",
    "(/ 1 (+ (% A B) (log (+ (% (log (+ A 2)) C) 3))))",
]


@pytest.mark.parametrize("tree", TREES)
def test_sigma_bounds_float32_rounding(tree):
    r = c = 48
    env = synth.operands(21, [("A", r, c), ("B", r, c), ("C", r, c), ("D", c, r), ("b", r, 1)],
                         "f32", "normal")
    R, C = np.arange(r)[:, None], np.arange(c)[None, :]
    z, s = oracle.at_sigma(tree, env, R, C)
    z32 = _f32_eval(tree, env, R, C).astype(np.float64)
    u = 2.0 ** -24
    ok = np.isfinite(z)
    assert np.all(np.abs(z32 - z)[ok] <= 4 * u * s[ok] + 1e-300)
    # the bound is not vacuous: it is within a few hundred u of |z| on average
    assert np.median(s[ok] / np.maximum(np.abs(z[ok]), 1e-30)) < 50


def _f32_product_tree(node, env):
    """Full-matrix FP32 evaluation where matrix products are summed in k
    order, one float32 rounding per multiply and per add (a plain loop over
    the inner dimension)."""
    n = oracle.parse(node)
    f = np.float32
    if n.op == "leaf":
        b = env[n.name]
        return oexpr._leaf_values(b, np.arange(b.rows)[:, None], np.arange(b.cols)[None, :]).astype(f)
    if n.op == "t":
        return _f32_product_tree(n.args[0], env).T.copy()
    if n.op == "*" and n.args[0].op == "num":
        return (f(n.args[0].value) * _f32_product_tree(n.args[1], env)).astype(f)
    if n.op == "*":
        A = _f32_product_tree(n.args[0], env)
        B = _f32_product_tree(n.args[1], env)
        acc = np.zeros((A.shape[0], B.shape[1]), dtype=f)
        for k in range(A.shape[1]):
            acc = (acc + (A[:, k:k + 1] * B[k:k + 1, :]).astype(f)).astype(f)
        return acc
    a = _f32_product_tree(n.args[0], env)
    b = _f32_product_tree(n.args[1], env)
    return {"+": lambda: a + b, "-": lambda: a - b, "%": lambda: a * b}[n.op]().astype(f)


@pytest.mark.parametrize("tree", ["(* 2 (* A (t D)))", "(* (* A B) C)",
                                  "(+ (* 0.5 (* A B)) C)", "(- (* (t D) B) A)"])
def test_sigma_bounds_float32_matrix_products(tree):
    """The product bound (K u |A||B| plus carried operand errors) covers a
    k-ordered FP32 summation, the worst order for a dot product."""
    r = 40
    env = synth.operands(23, [("A", r, r), ("B", r, r), ("C", r, r), ("D", r, r)], "f32",
                         "normal")
    z, s = oracle.evaluate_sigma(tree, env)
    z32 = _f32_product_tree(tree, env).astype(np.float64)
    u = 2.0 ** -24
    assert np.all(np.abs(z32 - z) <= 4 * u * s)
    assert np.all(s > 0)


def test_f32_conversion():
    """conv_to<fmat> (Sec. 4 expr3): round to nearest even into FP32."""
    vals = np.array([0.1, 1.0 + 2.0 ** -30, 1.0 + 3 * 2.0 ** -24, 2.0 ** 128, -2.5, 1e-46])
    env = {"Y": synth.Buffer(vals, 6, 1, 6, "f64")}
    got = oracle.evaluate("(f32 Y)", env)[:, 0]
    assert got[0] == 0.100000001490116119384765625          # nearest FP32 to 0.1
    assert got[1] == 1.0                                       # below half an ulp
    assert got[2] == 1.0 + 4 * 2.0 ** -24                      # tie at 1.5 ulp -> even (2 ulp)
    assert np.isinf(got[3]) and got[4] == -2.5 and got[5] == 0.0
    envf = synth.operands(5, [("X", 7, 3)], "f32", "normal")
    assert np.array_equal(oracle.evaluate("(f32 X)", envf), oracle.evaluate("X", envf))


def test_matrix_product_closed_forms():
    """ones(n, k) * ones(k, m) = k everywhere, with sigma = k * k; (A B)^T =
    B^T A^T exactly in FP64 for small integers."""
    n, k, m = 6, 9, 5
    env = {"O1": synth.Buffer(np.ones(n * k), n, k, n, "f64"),
           "O2": synth.Buffer(np.ones(k * m), k, m, k, "f64")}
    z, s = oracle.evaluate_sigma("(* O1 O2)", env)
    assert np.all(z == k) and np.all(s == k * k)
    rng = np.random.default_rng(3)
    env2 = {"A": synth.Buffer(rng.integers(-9, 10, 4 * 7).astype(np.float64), 4, 7, 4, "f64"),
            "B": synth.Buffer(rng.integers(-9, 10, 7 * 3).astype(np.float64), 7, 3, 7, "f64")}
    ab_t = oracle.evaluate("(t (* A B))", env2)
    bt_at = oracle.evaluate("(* (t B) (t A))", env2)
    assert np.array_equal(ab_t, bt_at)
    # brute-force triple loop
    A = env2["A"].data.reshape(7, 4).T
    B = env2["B"].data.reshape(3, 7).T
    ab = oracle.evaluate("(* A B)", env2)
    for i in range(4):
        for j in range(3):
            assert ab[i, j] == sum(A[i, q] * B[q, j] for q in range(7))


def test_sigma_reduction_rules():
    env = synth.operands(22, [("A", 40, 30), ("B", 40, 30)], "f32", "normal")
    v, s = oracle.evaluate_sigma("(accu (% A B))", env)
    prod = np.abs(env["A"].f64() * env["B"].f64())
    assert s[0, 0] == pytest.approx(2 * prod.sum(), rel=1e-12)
    v, s = oracle.evaluate_sigma("(max (abs (- A B)) 1)", env)
    assert np.allclose(s, v, rtol=1e-15)


# ------------------------------------------------------------ magnitude scale m

def test_magnitude_scale_by_hand():
    """m evaluates the tree on magnitudes: |a|+|b| for a sum or difference,
    |a||b| for a Schur product, |s||a| for a scalar, square of the
    magnitude; worked on a 2 x 2 case with mixed signs."""
    X = buf([1.0, -2.0, 3.0, -4.0], 2, 2)
    Y = buf([-0.5, 0.25, 2.0, -8.0], 2, 2)
    env = {"X": X, "Y": Y}
    R, C = np.arange(2)[:, None], np.arange(2)[None, :]
    ax = np.array([[1.0, 3.0], [2.0, 4.0]])
    ay = np.array([[0.5, 2.0], [0.25, 8.0]])
    assert np.array_equal(oracle.at_mag("(- X Y)", env, R, C), ax + ay)
    assert np.array_equal(oracle.at_mag("(+ X Y)", env, R, C), ax + ay)
    assert np.array_equal(oracle.at_mag("(% X Y)", env, R, C), ax * ay)
    assert np.array_equal(oracle.at_mag("(* -3 X)", env, R, C), 3 * ax)
    assert np.array_equal(oracle.at_mag("(square (- X Y))", env, R, C), (ax + ay) ** 2)
    assert np.array_equal(oracle.at_mag("(abs (neg X))", env, R, C), ax)
    # X - X is exactly 0, but its scale is 2|X|: a cancellation is visible in m
    assert np.all(oracle.evaluate("(- X X)", env) == 0)
    assert np.array_equal(oracle.at_mag("(- X X)", env, R, C), 2 * ax)
    # the transposed leaf maps positions the same way as the value rule
    assert np.array_equal(oracle.at_mag("(+ (t X) Y)", env, R, C), ax.T + ay)
    # the mask is exact: its scale is its value
    assert np.array_equal(oracle.at_mag("(% X (gt X 0))", env, R, C), ax * (np.array(
        [[1.0, 1.0], [0.0, 0.0]])))


def test_magnitude_scale_reductions_closed_forms():
    env = synth.operands(24, [("X", 37, 23), ("Y", 37, 23)], "f64", "normal")
    x, y = (np.abs(env[k].f64().reshape(23, 37).T) for k in "XY")
    m = x + y
    assert oracle.evaluate_mag("(accu (- X Y))", env)[0, 0] == pytest.approx(
        math.fsum(m.ravel()), rel=1e-15)
    assert oracle.evaluate_mag("(norm (- X Y))", env)[0, 0] == pytest.approx(
        math.sqrt(math.fsum((m * m).ravel())), rel=1e-15)
    assert np.allclose(oracle.evaluate_mag("(sum (% X Y) 0)", env)[0], (x * y).sum(axis=0),
                       rtol=1e-14, atol=0)
    assert np.allclose(oracle.evaluate_mag("(sum (% X Y) 1)", env)[:, 0], (x * y).sum(axis=1),
                       rtol=1e-14, atol=0)
    assert np.array_equal(oracle.evaluate_mag("(max (abs (- X Y)) 1)", env)[:, 0],
                          m.max(axis=1))
    assert np.array_equal(oracle.evaluate_mag("(max (abs (- X Y)) 0)", env)[0], m.max(axis=0))


M_TREES = ["(+ (+ (+ A B) C) (t D))", "(- (+ A C) (+ B C))", "(+ (% A B) (* 0.5 (t D)))",
           "(% (+ A B) (- C (t D)))", "(% A (gt A 0))", "(- (square (- A B)) (abs C))"]


@pytest.mark.parametrize("tree", M_TREES)
def test_magnitude_scale_bounds_float32_rounding(tree):
    """For trees of sums, products and scalars, a step-by-step FP32
    evaluation errs by a few u m; the scale never falls below |value|."""
    r = c = 48
    env = synth.operands(25, [("A", r, c), ("B", r, c), ("C", r, c), ("D", c, r)], "f32",
                         "normal")
    # C large against A and B: (A + C) - (B + C) cancels to about A - B
    env["C"].data[:] = (env["C"].data * 1000).astype(np.float32)
    R, C = np.arange(r)[:, None], np.arange(c)[None, :]
    z = oracle.at(tree, env, R, C)
    m = oracle.at_mag(tree, env, R, C)
    z32 = _f32_eval(tree, env, R, C).astype(np.float64)
    u = 2.0 ** -24
    assert np.all(m >= np.abs(z))
    assert np.all(np.abs(z32 - z) <= 4 * u * m + 1e-300)
    if tree == "(- (+ A C) (+ B C))":
        # a scale of |value| alone (no magnitude of the cancelled terms)
        # would not bound that evaluation
        assert np.any(np.abs(z32 - z) > 4 * u * np.abs(z))


def test_gate_scale_rule():
    from oracle.compare import gate_scale
    for t in ("(+ A B)", "(accu (square (- A B)))", "(sum (% X Y) 0)", "(max (abs (- X Y)) 1)",
              "(norm (- X Y))", "(% X (gt X 0))", "(+ (* 2 (+ (t X) Y)) (* 2 (+ X (t Y))))"):
        assert gate_scale(t) == "m", t
    for t in ("(- (+ (% A B) (* 3.5 (exp C))) (t D))", "(/ X (+ 1 (exp (neg X))))",
              "(sigmoid (+ (* 0.5 (* X Y)) W))", "(* 2 (* X (t Y)))", "(log (pow D 2))",
              "(/ A B)"):
        assert gate_scale(t) == "sigma", t


# ------------------------------------------------------------ gradient

LOSS = "(accu (square (- (sigmoid (+ (% X W) (each_col b))) Y)))"


def _fd_check(tree, env, names, rel=1e-6):
    g = oracle.gradient(tree, env)
    for name in names:
        b = env[name]
        for r in range(b.rows):
            for c in range(b.cols):
                k = r + c * b.ld
                x0 = float(b.data[k])
                h = 1e-6 * max(1.0, abs(x0))
                b.data[k] = x0 + h
                fp = oracle.evaluate(tree, env)[0, 0]
                b.data[k] = x0 - h
                fm = oracle.evaluate(tree, env)[0, 0]
                b.data[k] = x0
                fd = (fp - fm) / (2 * h)
                assert g[name][r, c] == pytest.approx(fd, rel=rel, abs=1e-8), (tree, name, r, c)


def test_gradient_loss_finite_differences():
    env = synth.operands(3, [("X", 6, 5), ("W", 6, 5), ("Y", 6, 5), ("b", 6, 1)], "f64",
                         "normal_half")
    _fd_check(LOSS, env, ["X", "W", "Y", "b"])


def test_gradient_loss_closed_form():
    env = synth.operands(3, [("X", 6, 5), ("W", 6, 5), ("Y", 6, 5), ("b", 6, 1)], "f64",
                         "normal_half")
    X, W, Y = (env[k].f64().reshape(5, 6).T for k in "XWY")
    bb = env["b"].f64()[:, None]
    S = 1 / (1 + np.exp(-(X * W + bb)))
    G = 2 * (S - Y) * S * (1 - S)
    g = oracle.gradient(LOSS, env, gL=0.75)
    assert np.allclose(g["X"], 0.75 * G * W, rtol=1e-14, atol=1e-16)
    assert np.allclose(g["W"], 0.75 * G * X, rtol=1e-14, atol=1e-16)
    assert np.allclose(g["b"][:, 0], 0.75 * G.sum(1), rtol=1e-13, atol=1e-16)
    # W = 0: U = b, so dX = G % 0 = 0 exactly
    env["W"].data[:] = 0.0
    assert np.all(oracle.gradient(LOSS, env)["X"] == 0.0)


@pytest.mark.parametrize("tree", [
    "(accu (exp (neg X)))", "(accu (log (+ (square X) 1)))", "(accu (sqrt (+ (abs X) 1)))",
    "(accu (tanh (% X Y)))", "(accu (/ X (+ 2 (square Y))))", "(accu (pow (+ X 3) 3))",
    "(accu (- (t X) (* 3 Y)))", "(accu (% (each_row r) (t X)))", "(accu (% X (gt X 0)))",
    "(accu (+ (* 2 (+ (t X) Y)) (* 2 (+ X (t Y)))))",
])
def test_gradient_ops_finite_differences(tree):
    env = synth.operands(13, [("X", 4, 4), ("Y", 4, 4), ("r", 1, 4)], "f64", "normal")
    if "gt" in tree:
        env["X"].data[np.abs(env["X"].data) < 1e-3] = 0.5      # stay off the kink
    names = [n for n in oracle.leaves_of(tree)]
    _fd_check(tree, env, names)


def test_gradient_rows_matches_full():
    env = synth.operands(3, [("X", 9, 7), ("W", 9, 7), ("Y", 9, 7), ("b", 9, 1)], "f64",
                         "normal_half")
    full = oracle.gradient(LOSS, env, gL=1.5)
    rows = [0, 4, 8]
    part = oracle.gradient_rows(LOSS, env, rows, gL=1.5)
    for name in ("X", "W", "Y", "b"):
        idx, val = part[name]
        b = env[name]
        for k, v in zip(idx.tolist(), val.tolist()):
            r, c = k % b.ld, k // b.ld
            assert r in rows
            assert v == pytest.approx(full[name][r, c], rel=1e-14, abs=1e-300)


# ------------------------------------------------------------ planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each mutation of the oracle must break at least one pin above."""
    f, expect = _read_golden("worked_example_trans_plus_scalar.txt")
    X = buf(f["data"], 2, 3)

    def worked_example_holds():
        return np.array_equal(oracle.evaluate("(+ (t X) 3)", {"X": X}), expect)

    def series_holds():
        env = {"X": buf(np.arange(60, dtype=np.float64), 6, 10)}
        return (oracle.evaluate("(accu X)", env)[0, 0] == 60 * 59 / 2
                and np.array_equal(oracle.evaluate("(sum X 0)", env)[0],
                                   np.arange(10) * 36.0 + 15.0))

    assert worked_example_holds() and series_holds()
    real = oexpr._leaf_values
    # 1. row-major storage rule (row*cols + col) instead of row + col*ld
    def row_major(b, R, C):
        k = (np.asarray(R) * b.cols + np.asarray(C)) % b.data.size
        return synth.to_f64(b.data[k], b.storage)
    monkeypatch.setattr(oexpr, "_leaf_values", row_major)
    assert not worked_example_holds()
    monkeypatch.setattr(oexpr, "_leaf_values", real)
    # 2. a dropped compensation term in the sums
    from oracle import sums
    real_axis = sums.neumaier_axis

    def plain_axis(a, axis, state=None):
        s, c = real_axis(a, axis, state)
        return s, np.zeros_like(c)
    monkeypatch.setattr(oexpr, "neumaier_axis", plain_axis)
    env = {"X": buf(np.array([1e16, 1.0, -1e16, 1.0]), 1, 4)}
    assert oracle.evaluate("(accu X)", env)[0, 0] != 2.0
    monkeypatch.setattr(oexpr, "neumaier_axis", real_axis)
    assert oracle.evaluate("(accu X)", env)[0, 0] == 2.0
    # 3. a wrong sign in the subtraction derivative
    from oracle import grad as ograd
    real_bp = ograd._backprop
    env = synth.operands(3, [("X", 3, 2), ("W", 3, 2), ("Y", 3, 2), ("b", 3, 1)], "f64",
                         "normal_half")
    good = oracle.gradient(LOSS, env)["Y"].copy()
    monkeypatch.setattr(ograd, "_unary_deriv", lambda op, a, z: oexpr._unary_deriv(op, a, z)
                        if op != "sigmoid" else z * (1.0 + z))
    bad = oracle.gradient(LOSS, env)["X"]
    monkeypatch.undo()
    assert not np.allclose(bad, oracle.gradient(LOSS, env)["X"])
    assert real_bp is ograd._backprop and np.array_equal(good, oracle.gradient(LOSS, env)["Y"])


def test_gradient_sigma_bounds_float32_reverse_pass():
    """The reverse-pass error bound holds for a step-by-step FP32 evaluation
    of the loss gradient (closed form of the same reverse pass)."""
    from oracle import grad as ograd
    r, c = 40, 30
    env = synth.operands(3, [("X", r, c), ("W", r, c), ("Y", r, c), ("b", r, 1)], "f32",
                         "normal_half")
    f = np.float32
    X, W, Y = (env[k].data.reshape(c, r).T for k in "XWY")
    b = env["b"].data[:, None]
    U = X * W + b
    S = f(1) / (f(1) + np.exp(-U))
    G = (f(2) * (S - Y)) * (S * (f(1) - S))
    g32 = {"X": G * W, "W": G * X, "Y": f(-2) * (S - Y), "b": G.sum(axis=1, dtype=np.float32)[:, None]}
    gs = ograd.gradient_sigma(LOSS, env)
    u = 2.0 ** -24
    for name in "XWYb":
        idx, v, s = gs[name]
        got = g32[name].T.ravel().astype(np.float64) if name != "b" else g32[name].ravel()
        assert np.all(np.abs(got - v) <= 8 * u * s + 1e-300), name
        assert np.median(s / np.maximum(np.abs(v), 1e-300)) < 100, name


# ------------------------------------------------------------ Sec. 4 trees of the suite

def _suite_tree(name, scalars=None):
    from harness import tree_of
    return tree_of(name, scalars)


def test_expr2_hand_values():
    """expr2 = a*A + (B + C)^T + log(pow(D, 2)) with the suite's a = 0.75 and
    exponent 2, on a 2x2 case worked by hand: 0.75*[[4,8],[12,16]] = [[3,6],[9,12]],
    ([[1,2],[3,4]] + [[10,20],[30,40]])^T = [[11,33],[22,44]], log(D^2) = 0 for
    D = +-1, so Z = [[14,39],[31,56]]; with D = e every element gains log(e^2) = 2."""
    tree = _suite_tree("expr2")
    A = buf([4, 12, 8, 16], 2, 2)
    B = buf([1, 3, 2, 4], 2, 2)
    C = buf([10, 30, 20, 40], 2, 2)
    got = oracle.evaluate(tree, {"A": A, "B": B, "C": C, "D": buf([1, -1, -1, 1], 2, 2)})
    assert got.T.ravel().tolist() == [14.0, 31.0, 39.0, 56.0]
    got = oracle.evaluate(tree, {"A": A, "B": B, "C": C, "D": buf([math.e] * 4, 2, 2)})
    assert np.allclose(got.T.ravel(), [16.0, 33.0, 41.0, 58.0], rtol=0, atol=1e-14)


@pytest.mark.parametrize("beta", [None, 2.5])
def test_swish_odd_part_is_x(beta):
    """swish(x) = x * sigmoid(beta x) (Sec. 4). Since sigmoid(t) + sigmoid(-t) = 1,
    swish(x) - swish(-x) = x for every beta, and swish(0) = 0."""
    tree = _suite_tree("swish", None if beta is None else [beta])
    x = np.linspace(-6.0, 6.0, 25)
    zp = oracle.evaluate(tree, {"X": buf(x, 25, 1)})[:, 0]
    zm = oracle.evaluate(tree, {"X": buf(-x, 25, 1)})[:, 0]
    assert np.allclose(zp - zm, x, rtol=0, atol=1e-14)
    assert zp[12] == 0.0
    assert np.all(zp[x > 0] > 0) and np.all(zp[x > 0] < x[x > 0])


def test_gelu_odd_part_limits_and_exact_gelu():
    """gelu = (x/2)(1 + tanh(s0 (x + s1 x^3))) (Sec. 4, s0 = sqrt(2/pi),
    s1 = 0.044715): tanh is odd, so gelu(x) - gelu(-x) = x; gelu(0) = 0; far
    out gelu(x) = x and gelu(-x) = 0. The tanh form approximates the exact
    GELU x * Phi(x) = (x/2)(1 + erf(x / sqrt 2)) to within 1e-3 (without the
    cubic term it is off by 0.03 at x = 2)."""
    tree = _suite_tree("gelu")
    x = np.linspace(-5.0, 5.0, 41)
    zp = oracle.evaluate(tree, {"X": buf(x, 41, 1)})[:, 0]
    zm = oracle.evaluate(tree, {"X": buf(-x, 41, 1)})[:, 0]
    assert np.allclose(zp - zm, x, rtol=0, atol=1e-14)
    assert zp[20] == 0.0
    far = oracle.evaluate(tree, {"X": buf([30.0, -30.0], 2, 1)})[:, 0]
    assert far[0] == 30.0 and far[1] == 0.0
    exact = np.array([0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0))) for v in x])
    assert np.max(np.abs(zp - exact)) < 1e-3
    no_cubic = oracle.evaluate(_suite_tree("gelu", [math.sqrt(2.0 / math.pi), 0.0]),
                               {"X": buf([2.0], 1, 1)})[0, 0]
    assert abs(no_cubic - 0.5 * 2.0 * (1.0 + math.erf(2.0 / math.sqrt(2.0)))) > 0.02


def test_expr3_reduces_to_reciprocal_product():
    """expr3 = 1 / (X % conv_to<fmat>(Y) + log(log(X + 2) % W)) (Sec. 4): with
    W = 1 / log(X + 2) the outer log vanishes and Z = 1 / (X * fl32(Y)); Y = 0.1
    is read as its nearest FP32 value 0.100000001490116119384765625."""
    tree = _suite_tree("expr3")
    X = np.array([10.0, 0.5, 3.0, 7.25])
    Y = np.array([0.1, 4.0, -0.75, 1.0 / 3.0])
    W = 1.0 / np.log(X + 2.0)
    got = oracle.evaluate(tree, {"X": buf(X, 4, 1), "Y": buf(Y, 4, 1), "W": buf(W, 4, 1)})[:, 0]
    want = 1.0 / (X * Y.astype(np.float32).astype(np.float64))
    assert np.allclose(got, want, rtol=1e-14, atol=0)
    assert got[0] != 1.0 / (X[0] * Y[0])       # the FP32 conversion of Y is visible


L3 = math.log(3.0)   # sigmoid(ln 3) = 1 / (1 + 1/3) = 3/4

# Each oracle tree the parity tests compare against (as tests/harness.py
# writes it, default scalars), on a small case worked by hand from the
# paper's definitions. Leaves: (column-major values, rows, cols).
HAND_TREES = {
    # A%B + 3.5*exp(C) - D^T: [[2,4],[6,8]] + 3.5 - [[0,2],[1,3]]
    "schur_exp_trans": ({"A": ([1, 3, 2, 4], 2, 2), "B": ([2, 2, 2, 2], 2, 2),
                         "C": ([0, 0, 0, 0], 2, 2), "D": ([0, 2, 1, 3], 2, 2)},
                        [5.5, 8.5, 5.5, 8.5]),
    # (A-B)^2 summed: 9 + 16
    "sqdiff_accu": ({"A": ([1, 2], 2, 1), "B": ([4, 6], 2, 1)}, [25.0]),
    # X%Y + sqrt(|W|)/(1 + exp(-V)): 6 + 4/2, 1 + 3/2
    "schur_sqrt_sigmoid": ({"X": ([2, 1], 2, 1), "Y": ([3, 1], 2, 1), "W": ([-16, 9], 2, 1),
                            "V": ([0, 0], 2, 1)}, [8.0, 2.5]),
    # column sums of [[1,2],[6,8]]
    "schur_colsum": ({"X": ([1, 3, 2, 4], 2, 2), "Y": ([1, 2, 1, 2], 2, 2)}, [7.0, 10.0]),
    # row maxima of |[[3,4],[1,7]] - [[2,-1],[-1,4]]| = [[1,5],[2,3]] (column maxima
    # would be 2, 5)
    "absdiff_rowmax": ({"X": ([3, 1, 4, 7], 2, 2), "Y": ([2, -1, -1, 4], 2, 2)}, [5.0, 3.0]),
    # |(3, 4)| = 5
    "diff_norm": ({"X": ([5, 5], 2, 1), "Y": ([2, 1], 2, 1)}, [5.0]),
    # A%B + 0.5*C^T: [[1,2],[3,4]] + [[1,3],[2,4]]
    "schur_trans_accu": ({"A": ([1, 3, 2, 4], 2, 2), "B": ([1, 1, 1, 1], 2, 2),
                          "C": ([2, 6, 4, 8], 2, 2)}, [2.0, 5.0, 5.0, 8.0]),
    # X%W = 0, so sigmoid(b_r) = 1/2 (row 0), 3/4 (row 1); residuals 0, .5, 0, -.25
    "sigmoid_sqloss": ({"X": ([0, 0, 0, 0], 2, 2), "W": ([7, -3, 2, 5], 2, 2),
                        "Y": ([0.5, 0.75, 0, 1], 2, 2), "b": ([0, L3], 2, 1)}, [0.3125]),
    # 2*(X^T + Y) + 2*(X + Y^T) with X = [[1,2],[3,4]], Y = [[0,1],[1,0]]
    "expr1": ({"X": ([1, 3, 2, 4], 2, 2), "Y": ([0, 1, 1, 0], 2, 2)}, [4.0, 14.0, 14.0, 16.0]),
    "relu": ({"X": ([-2, 0, 3.5, -0.25], 2, 2)}, [0.0, 0.0, 3.5, 0.0]),
    "sigmoid": ({"X": ([0, L3, -L3], 3, 1)}, [0.5, 0.75, 0.25]),
    # (1 + 2) * (3 + 4)
    "sum_schur": ({"A": ([1], 1, 1), "B": ([2], 1, 1), "C": ([3], 1, 1), "D": ([4], 1, 1)},
                  [21.0]),
    # 2 * X Y^T, X = [[1,2],[3,4]], Y = [[1,2],[0,1]]: X Y^T = [[5,2],[11,4]]
    # (X Y would be [[1,4],[3,10]])
    "gemm_scale": ({"X": ([1, 3, 2, 4], 2, 2), "Y": ([1, 0, 2, 1], 2, 2)},
                   [10.0, 22.0, 4.0, 8.0]),
    # sigmoid(0.5 X Y + W), X = [[2,2],[0,2]], Y = [[1,0],[-1,1]]: 0.5 X Y =
    # [[0,1],[-1,1]] (0.5 Y X would be [[1,1],[-1,0]]); + W = [[0, ln3], [-ln3, 0]]
    "gemm_epilogue": ({"X": ([2, 0, 2, 2], 2, 2), "Y": ([1, -1, 0, 1], 2, 2),
                       "W": ([0, 1 - L3, L3 - 1, -1], 2, 2)}, [0.5, 0.25, 0.75, 0.5]),
    # [[1,1],[0,1]] [[1,0],[1,1]] = [[2,1],[1,1]]; * [[0,1],[1,0]] = [[1,2],[1,1]];
    # * diag(1, 2) = [[1,4],[1,2]]
    "chain": ({"A": ([1, 0, 1, 1], 2, 2), "B": ([1, 1, 0, 1], 2, 2), "C": ([0, 1, 1, 0], 2, 2),
               "D": ([1, 0, 0, 2], 2, 2)}, [1.0, 1.0, 4.0, 2.0]),
}


@pytest.mark.parametrize("name", sorted(HAND_TREES))
def test_suite_trees_by_hand(name):
    from harness import tree_of
    leaves, want = HAND_TREES[name]
    env = {k: buf(v, r, c) for k, (v, r, c) in leaves.items()}
    got = np.asarray(oracle.evaluate(tree_of(name), env), dtype=np.float64)
    got = got.T.ravel() if got.ndim == 2 else got.ravel()
    assert np.allclose(got, want, rtol=0, atol=1e-15), (name, got, want)


@pytest.mark.parametrize("n", range(2, 17))
def test_add_n_of_index_matrices(n):
    """add-N over A_k = k * ones sums to n(n+1)/2 everywhere."""
    from harness import tree_of
    env = {f"A{k}": buf([float(k)] * 6, 2, 3) for k in range(1, n + 1)}
    got = oracle.evaluate(tree_of(f"add{n}"), env)
    assert np.all(got == n * (n + 1) / 2)
