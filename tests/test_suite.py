"""The Sec. 4 expression suite on the fused path (GPU): add-N for N = 2..16,
expr1, expr2, relu, sigmoid, swish, gelu, and the view-based cases
addsub2/addsub4 (submatrix leaves) and diagsum (diagonal leaves)."""
import numpy as np
import pytest

import synth
from harness import oracle_outputs, panel_report, record, run, scaled_error, specs_for, tolerance

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (33, 17), (64, 64), (100, 37), (257, 129)]
SQUARE = [(1, 1), (33, 33), (64, 64), (100, 100), (257, 257)]


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


def check(name, got, env, label, scalars=None):
    for key, (rv, rs) in oracle_outputs(name, env, scalars).items():
        tol = tolerance(name, "f32", key)
        err, _, bad, _ = scaled_error(got[key], rv, rs, "f32")
        assert bad == 0, f"{name}{label}: {bad} wrong non-finite outputs"
        assert err <= tol, f"{name}{label}: scaled error {err:.3e} > {tol:.1e}"


@pytest.mark.parametrize("n", list(range(2, 17)))
def test_add_n(fx, n):
    name = f"add{n}"
    for R, C in SHAPES:
        env = synth.operands(40 + n, specs_for(name, R, C), "f32", "uniform")
        got = run(fx, name, "f32", env, R, C)
        check(name, got, env, f" at {R}x{C}")
        assert got["_launches"] == 1


@pytest.mark.parametrize("n", [2, 9, 16])
def test_add_n_bulk_copies(fx, n):
    """The bulk-copy flat kernel (pipeline 1): several chunks per block, a
    last chunk shorter than the rest and elements after the last whole
    16-byte vector; one and two CTAs per SM; and the register kernel
    (pipeline 2) on the same trees."""
    name = f"add{n}"
    for R, C in [(1000, 700), (333, 129), (64, 64), (5, 3)]:
        env = synth.operands(60 + n, specs_for(name, R, C), "f32", "uniform")
        for shape in [(256, 4, 0, 1), (256, 4, 1, 1), (256, 4, 2, 1), (256, 2, 0, 2)]:
            got = run(fx, name, "f32", env, R, C, shape=shape)
            check(name, got, env, f" at {R}x{C} shape {shape}")
            assert got["_launches"] == 1


@pytest.mark.parametrize("name", ["expr1", "expr2", "relu", "sigmoid", "swish", "gelu"])
def test_suite_expressions(fx, name):
    shapes = SQUARE if name == "expr1" else SHAPES
    for R, C in shapes:
        env = synth.operands(50, specs_for(name, R, C), "f32", "normal")
        got = run(fx, name, "f32", env, R, C)
        check(name, got, env, f" at {R}x{C}")


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
def test_expr1_symmetric_tile_pairs(fx, storage):
    """expr1 reads X and Y both plain and transposed, so on the TMA kernel
    (launch-shape pipeline 0) one work item is the tile pair {(i, j), (j, i)}:
    the four boxes are loaded once and both output tiles are written. Square
    sizes from one tile to many, with and without a ragged last tile (64 and
    32 elements per tile side), a padded output, one and two CTAs per SM;
    every element against the oracle."""
    for n in [8, 64, 72, 136, 1000]:
        env = synth.operands(70 + n, specs_for("expr1", n, n), storage, "normal")
        for shape, ldz in [((256, 4, 0, 0), None), ((256, 4, 1, 0), n + 8), ((256, 4, 2, 0), None)]:
            got = run(fx, "expr1", storage, env, n, n, shape=shape, ldz=ldz)
            for key, (rv, rs) in oracle_outputs("expr1", env).items():
                tol = tolerance("expr1", storage, key)
                err, _, bad, _ = scaled_error(got[key], rv, rs, storage)
                assert bad == 0, f"expr1 {storage} {n}^2 {shape}: {bad} wrong non-finite outputs"
                assert err <= tol, f"expr1 {storage} {n}^2 {shape}: {err:.3e} > {tol:.1e}"
            assert got["_launches"] == 1


@pytest.mark.parametrize("name", ["add5", "sum_schur", "relu"])
def test_lane_pairs_round_like_scalar_lanes(fx, name):
    """FP32 trees run on lane pairs (add/sub/mul.rn.f32x2) when their
    operands are 16-byte aligned and lane by lane when they are not (inputs
    one element off alignment take the one-lane path). Trees of adds and
    multiplies only, with no product added to something (where the two
    paths may contract differently), must agree bit for bit."""
    for R, C in [(333, 129), (64, 64), (1000, 7)]:
        env = synth.operands(80, specs_for(name, R, C), "f32", "normal")
        paired = run(fx, name, "f32", env, R, C)
        single = run(fx, name, "f32", env, R, C, offset=1)
        assert np.array_equal(paired["Z"], single["Z"]), f"{name} at {R}x{C}"


def expr3_env(seed, R, C):
    """expr3's inputs: X and W positive FP32 (the logs stay defined), Y FP64."""
    env = synth.operands(seed, [("X", R, C), ("W", R, C)], "f32", "positive")
    env.update(synth.operands(seed + 1, [("Y", R, C)], "f64", "normal"))
    return env


def test_expr3_mixed_storage(fx):
    """Sec. 4 expr3: an FP64 leaf in an FP32 tree, read as its FP32 rounding."""
    h = fx.fx_expr_create("expr3", fx.FX_F32)
    try:
        assert [fx.fx_expr_slot_dtype(h, k) for k in range(4)] == [fx.FX_F32, fx.FX_F64, fx.FX_F32,
                                                                   fx.FX_F32]
    finally:
        fx.fx_expr_destroy(h)
    for R, C in SHAPES + [(1000, 700)]:
        env = expr3_env(110, R, C)
        got = run(fx, "expr3", "f32", env, R, C)
        check("expr3", got, env, f" at {R}x{C}")
        assert got["_launches"] == 1


def _submatrix(parent, r0, c0, rows, cols):
    """A view of `parent` (a synth.Buffer): pointer offset, the parent's ld."""
    off = r0 + c0 * parent.ld
    return synth.Buffer(parent.data[off:], rows, cols, parent.ld, parent.storage)


@pytest.mark.parametrize("n", [2, 4])
def test_addsub_views(fx, n):
    # the centre of each matrix with half the rows and columns
    P = 96
    parents = synth.operands(60, [(f"A{k}", P, P) for k in range(1, n + 1)], "f32", "uniform")
    env = {k: _submatrix(b, P // 4, P // 4, P // 2, P // 2) for k, b in parents.items()}
    got = run(fx, f"add{n}", "f32", env, P // 2, P // 2)
    check(f"add{n}", got, env, " (centre submatrices)")


def test_diagsum_views(fx):
    # (X.diag(-1) + X.diag(1)) % (Y.diag(-1) + Y.diag(1)) as 1 x (n-1) leaves
    n = 130
    XY = synth.operands(61, [("X", n, n), ("Y", n, n)], "f32", "normal")

    def diag(b, k):
        off = -k if k < 0 else k * b.ld      # element (-k, 0) or (0, k)
        return synth.Buffer(b.data[off:], 1, n - 1, b.ld + 1, b.storage)

    env = {"A": diag(XY["X"], -1), "B": diag(XY["X"], 1), "C": diag(XY["Y"], -1),
           "D": diag(XY["Y"], 1)}
    got = run(fx, "sum_schur", "f32", env, 1, n - 1)
    check("sum_schur", got, env, " (diagonal views)")
    X = XY["X"].f64().reshape(n, n).T
    Y = XY["Y"].f64().reshape(n, n).T
    want = (np.diag(X, -1) + np.diag(X, 1)) * (np.diag(Y, -1) + np.diag(Y, 1))
    assert np.allclose(got["Z"][0], want, rtol=1e-6, atol=1e-6)


def test_unfused_suite(fx):
    for name in ["add8", "expr1", "expr2", "gelu"]:
        R = C = 64
        env = synth.operands(62, specs_for(name, R, C), "f32", "normal")
        got = run(fx, name, "f32", env, R, C, unfused=True)
        check(name, got, env, " (unfused)")


# ---------------------------------------------------------------- Sec. 4 sizes

@pytest.fixture(scope="module")
def suite10k():
    """The benchmark's 10000^2 FP32 inputs: A1..A16 U[-1, 1] (seed 4); P1, P2
    U[0.5, 2] (seed 5) and Y64 FP64 N(0, 1) (seed 6) for expr3."""
    R = C = 10000
    env = synth.operands(4, [(f"A{k}", R, C) for k in range(1, 17)], "f32", "uniform")
    env.update(synth.operands(5, [("P1", R, C), ("P2", R, C)], "f32", "positive"))
    env.update(synth.operands(6, [("Y64", R, C)], "f64", "normal"))
    return env


# the benchmark's binding of those inputs to each tree's slots
BENCH_INPUTS = {"add16": [f"A{k}" for k in range(1, 17)], "expr1": ["A1", "A2"],
                "expr2": ["A1", "A2", "A3", "A4"], "expr3": ["P1", "Y64", "P2"], "gelu": ["A1"]}


@pytest.mark.parametrize("name", ["add16", "expr1", "expr2", "expr3", "gelu"])
def test_suite_10000_autotuned(fx, suite10k, name):
    """The Sec. 4 expressions at the paper's 10000^2 size, autotuned as the
    benchmark runs them, every output element against the oracle."""
    from harness import SLOTS
    R = C = 10000
    env = {slot: suite10k[src] for slot, src in zip(SLOTS[name], BENCH_INPUTS[name])}
    got = run(fx, name, "f32", env, R, C, tune="search")
    rep = panel_report(name, "f32", got["Z"], env)
    record(f"{name}/f32/Z at 10000^2 (shape {got['_shape']})", rep)
    assert rep.nonfinite == 0
    assert rep.err <= rep.tol, f"{name} at 10000^2: scaled error {rep.err:.3e} > {rep.tol:.1e}"
    assert rep.n == R * C
