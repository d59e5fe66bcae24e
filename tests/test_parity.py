"""Parity of the fused CUDA path with the FP64 oracle (GPU).

Small and ragged shapes, and the full-size workloads (1024^2 FP32, 8192^2
FP32/FP64, 16384^2 BF16/FP16 on the benchmark's own seeds, each tree
autotuned first as the benchmark does), compared element by element.
"""
import numpy as np
import pytest

import oracle
import synth
from harness import (SLOTS, oracle_outputs, panel_report, record, run, scaled_error, specs_for,
                     tolerance, tree_of)

pytestmark = pytest.mark.gpu

NAMES = ["schur_exp_trans", "sqdiff_accu", "schur_exp_trans_sqdiff", "schur_sqrt_sigmoid",
         "schur_colsum", "absdiff_rowmax", "diff_norm", "schur_trans_accu", "sigmoid_sqloss"]
DIST = {"schur_exp_trans": "uniform", "sqdiff_accu": "uniform", "schur_trans_accu": "uniform",
        "schur_exp_trans_sqdiff": "uniform", "sigmoid_sqloss": "normal_half"}
SMALL = [(1, 1), (1, 7), (7, 1), (33, 17), (100, 37), (257, 129), (64, 64)]


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


def check(name, storage, got, ref, label=""):
    for key, (rv, rs) in ref.items():
        tol = tolerance(name, storage, key)
        # reductions are stored in FP32 (FP64 for f64)
        st = storage if key == "Z" else ("f64" if storage == "f64" else "f32")
        err, nover, bad, rel = scaled_error(got[key], rv, rs, st)
        assert bad == 0, f"{name}/{storage}/{key}{label}: {bad} wrong non-finite outputs"
        assert err <= tol, f"{name}/{storage}/{key}{label}: scaled error {err:.3e} > {tol:.1e}"


def env_for(name, storage, R, C, seed=7, lds=None):
    return synth.operands(seed, specs_for(name, R, C), storage, DIST.get(name, "normal"), lds=lds)


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("name", NAMES)
def test_small_shapes(fx, name, storage):
    for R, C in SMALL:
        env = env_for(name, storage, R, C)
        got = run(fx, name, storage, env, R, C)
        check(name, storage, got, oracle_outputs(name, env), f" at {R}x{C}")


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("name", NAMES)
def test_leading_dimension_and_misalignment(fx, name, storage):
    R, C = 45, 23
    lds = {s: (c_rows + 3) for s, c_rows, _ in specs_for(name, R, C)}
    env = env_for(name, storage, R, C, seed=11, lds=lds)
    ref = oracle_outputs(name, env)
    check(name, storage, run(fx, name, storage, env, R, C, ldz=R + 5), ref, " (ld > rows)")
    env2 = env_for(name, storage, R, C, seed=12)
    ref2 = oracle_outputs(name, env2)
    check(name, storage, run(fx, name, storage, env2, R, C, offset=1), ref2, " (misaligned base)")


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("name", NAMES)
def test_unfused_baseline_matches(fx, name, storage):
    R, C = 96, 80
    env = env_for(name, storage, R, C, seed=13)
    got = run(fx, name, storage, env, R, C, unfused=True)
    check(name, storage, got, oracle_outputs(name, env), " (unfused)")
    assert got["_launches"] >= 2


@pytest.mark.parametrize("name", ["sqdiff_accu", "schur_colsum", "absdiff_rowmax", "diff_norm",
                                  "schur_trans_accu", "sigmoid_sqloss", "schur_exp_trans_sqdiff"])
def test_reductions_bitwise_repeatable(fx, name):
    R, C = 1000, 700
    env = env_for(name, "f32", R, C, seed=14)
    a = run(fx, name, "f32", env, R, C)
    b = run(fx, name, "f32", env, R, C)
    for k in a:
        if k != "_launches":
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


# Launch shapes: every kernel variant (transposed tiles by TMA, cp.async or
# registers; dim-1 rows by bulk copies or registers), small and large
# blocks, shallow and deep unrolling, capped residency. Shapes span several
# tiles, split columns and ragged tails.
SHAPES = [(256, 4, 0, 1), (128, 2, 2, 1), (512, 8, 0, 0), (64, 2, 1, 2), (256, 8, 4, 2)]


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("name", NAMES)
def test_launch_shapes(fx, name, storage):
    for i, shape in enumerate(SHAPES):
        for R, C in [(257, 129), (1000, 700), (64, 64)]:
            env = env_for(name, storage, R, C, seed=20 + i)
            got = run(fx, name, storage, env, R, C, shape=shape)
            check(name, storage, got, oracle_outputs(name, env), f" at {R}x{C} shape {shape}")


@pytest.mark.parametrize("name", ["schur_exp_trans", "schur_trans_accu", "absdiff_rowmax",
                                  "schur_exp_trans_sqdiff"])
def test_kernel_variants_agree_bitwise(fx, name):
    """Every variant evaluates an element with the same operations, so the
    element-wise outputs and the row maxima agree bit for bit."""
    R, C = 1500, 900
    env = env_for(name, "f32", R, C, seed=31)
    outs = [run(fx, name, "f32", env, R, C, shape=(256, 4, 0, p)) for p in (0, 1, 2)]
    key = "Z" if "Z" in outs[0] else "v"
    for o in outs[1:]:
        assert np.array_equal(outs[0][key], o[key])


# Shapes whose leading dimensions TMA can address (multiples of 16 bytes):
# ragged last tiles, last tiles whose second box starts outside the matrix
# (972 rows in FP32: boxes at 960 and 992; 970 rows in FP64: 960 and 976;
# 712 columns: 704 and 736), and a single full tile.
TMA_SHAPES = {"f32": [(1000, 700), (972, 712), (64, 64)], "bf16": [(1000, 712), (968, 136)],
              "f16": [(1000, 712)], "f64": [(1000, 702), (970, 98)]}


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("name", ["schur_exp_trans", "schur_trans_accu", "schur_exp_trans_sqdiff"])
def test_tma_tiles(fx, name, storage):
    for k, (R, C) in enumerate(TMA_SHAPES[storage]):
        env = env_for(name, storage, R, C, seed=40 + k)
        ref = oracle_outputs(name, env)
        for pipe in (0, 1, 2):
            got = run(fx, name, storage, env, R, C, shape=(256, 4, 0, pipe))
            check(name, storage, got, ref, f" at {R}x{C} pipeline {pipe}")
        got = run(fx, name, storage, env, R, C, shape=(256, 4, 2, 0))
        check(name, storage, got, ref, f" at {R}x{C} two blocks per SM")
    # padded leading dimensions, still 16-byte multiples, on leaves and output
    R, C = 520, 264
    lds = {s: rows + 8 for s, rows, _ in specs_for(name, R, C)}
    env = env_for(name, storage, R, C, seed=49, lds=lds)
    got = run(fx, name, storage, env, R, C, ldz=R + 8, shape=(256, 4, 0, 0))
    check(name, storage, got, oracle_outputs(name, env), " (padded leading dimensions)")


def test_launch_shape_rejects_bad_values(fx):
    h = fx.fx_expr_create("schur_exp_trans", 0)
    try:
        before = fx.fx_expr_launch_shape(h)
        for bad in [(48, 4, 0, 0), (256, 3, 0, 0), (256, 4, -1, 0), (256, 4, 0, 3), (1024, 4, 0, 0)]:
            with pytest.raises(fx.FxError):
                fx.fx_expr_set_launch_shape(h, *bad)
            assert fx.fx_expr_launch_shape(h) == before
    finally:
        fx.fx_expr_destroy(h)


def test_one_launch_per_fused_tree(fx):
    for name in NAMES:
        env = env_for(name, "f32", 300, 200)
        assert run(fx, name, "f32", env, 300, 200)["_launches"] == 1, name


@pytest.mark.parametrize("name", NAMES)
def test_empty_shapes(fx, name):
    for R, C in [(0, 5), (5, 0), (0, 0)]:
        env = env_for(name, "f32", R, C)
        got = run(fx, name, "f32", env, R, C)
        if "s" in got:
            assert got["s"] == 0.0
        if "v" in got:
            if name == "absdiff_rowmax":
                assert np.all(got["v"] == -np.inf)
            else:
                assert np.all(got["v"] == 0.0)


def test_scalar_override(fx):
    R, C = 50, 40
    env = env_for("schur_exp_trans", "f32", R, C)
    got = run(fx, "schur_exp_trans", "f32", env, R, C, scalars=[-0.75])
    check("schur_exp_trans", "f32", got, oracle_outputs("schur_exp_trans", env, [-0.75]))


# ---------------------------------------------------------------- full-size workloads
#
# The configurations the benchmark times, on its own inputs (the same seeds
# and distributions), each tree autotuned first as the benchmark does, and
# every output element compared with the oracle (column panels evaluated on
# a thread pool).

def full_check(fx, name, storage, env, R, C, label):
    got = run(fx, name, storage, env, R, C, tune="search")
    reports = {}
    if "Z" in got:
        rep = panel_report(name, storage, got["Z"], env)
        record(f"{name}/{storage}/Z{label}", rep)
        assert rep.nonfinite == 0, f"{name}/{storage}/Z{label}: {rep.nonfinite} wrong non-finite"
        assert rep.err <= rep.tol, f"{name}/{storage}/Z{label}: scaled error {rep.err:.3e}"
        assert rep.n == R * C
        reports["Z"] = rep
    red = {k: v for k, v in got.items() if k in ("s", "v")}
    if red:
        ref = {k: v for k, v in oracle_outputs(name, env).items() if k in red}
        check(name, storage, red, ref, label)
    return reports


def test_workload_1024_f32(fx):
    R = C = 1024
    env = synth.operands(0, [("A", R, C), ("B", R, C), ("C", R, C), ("D", C, R)], "f32", "uniform")
    for name in ("schur_exp_trans_sqdiff", "schur_exp_trans", "sqdiff_accu"):
        full_check(fx, name, "f32", env, R, C, " at 1024^2")


def test_two_results_match_the_separate_trees(fx):
    """Z and s of the one-pass definition are bit for bit those of the two
    separate trees: Z's elements take the same operations, and the sum runs
    over the same values (the launch shapes are fixed alike; the grids, and
    so the partial sums' grouping, can differ, so s is held to the
    reduction bound instead)."""
    R, C = 1000, 712
    env = synth.operands(3, [("A", R, C), ("B", R, C), ("C", R, C), ("D", C, R)], "f32", "uniform")
    for pipe in (0, 1, 2):
        both = run(fx, "schur_exp_trans_sqdiff", "f32", env, R, C, shape=(256, 4, 0, pipe))
        z = run(fx, "schur_exp_trans", "f32", env, R, C, shape=(256, 4, 0, pipe))
        s = run(fx, "sqdiff_accu", "f32", env, R, C, shape=(256, 4, 0, pipe))
        assert np.array_equal(both["Z"], z["Z"]), pipe
        assert abs(both["s"] - s["s"]) <= 1e-6 * abs(s["s"]), pipe
        assert both["_launches"] == 1


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_workload_8192(fx, storage):
    R = C = 8192
    env = synth.operands(1, [("X", R, C), ("Y", R, C), ("W", R, C), ("V", R, C)], storage,
                         "normal")
    for name in ("schur_sqrt_sigmoid", "schur_colsum", "absdiff_rowmax", "diff_norm"):
        full_check(fx, name, storage, env, R, C, " at 8192^2")


@pytest.fixture(scope="module", params=["bf16", "f16"])
def env16384(request):
    """The precision workload's inputs: A, B, C, D (D transposed) at 16384^2,
    +-lognormal(0, 1), seed 0 (the seed of the 1024^2 workload, whose trees
    these are)."""
    R = C = 16384
    storage = request.param
    return storage, synth.operands(0, [("A", R, C), ("B", R, C), ("C", R, C), ("D", C, R)],
                                   storage, "lognormal_signed")


def test_workload_16384(fx, env16384):
    storage, env = env16384
    R = C = 16384
    reps = {}
    reps.update(full_check(fx, "schur_exp_trans_sqdiff", storage, env, R, C, " at 16384^2"))
    # 3.5 exp(C) passes the FP16 maximum (65504) for C > 9.84: such outputs
    # must be infinities of the oracle's sign (checked above); there are some
    over = reps["Z"].overflow
    if storage == "f16":
        assert over > 0, "the FP16 run should exercise overflowing outputs"


def test_workload_16384_clamped(fx, env16384):
    """The same trees with C's values capped at 9 (3.5 exp(9) = 28361 is
    finite in FP16), so every FP16 output has a finite comparison."""
    storage, env = env16384
    R = C = 16384
    cap = synth.round_to_storage(np.array([9.0]), storage)[0]
    c = env["C"]
    vals = synth.to_f64(c.data, storage)
    clamped = synth.Buffer(np.where(vals > 9.0, cap, c.data), c.rows, c.cols, c.ld, storage)
    env2 = dict(env, C=clamped)
    rep = full_check(fx, "schur_exp_trans_sqdiff", storage, env2, R, C, " at 16384^2, C <= 9")["Z"]
    assert rep.overflow == 0


@pytest.mark.parametrize("name", ["sqdiff_accu", "diff_norm", "absdiff_rowmax", "schur_colsum",
                                  "schur_trans_accu", "schur_exp_trans_sqdiff", "sigmoid_sqloss"])
def test_alternating_evaluations_on_one_object(fx, name):
    """One expression object evaluated fused, unfused and fused again under
    launch shapes with different grids (so the partial sums are laid out
    differently each time): every result is complete and correct. The
    combines' completion tickets live apart from the partials."""
    import torch
    from harness import STORAGE_CODE, canary_buffer, from_device, to_device
    R, C = 1000, 700
    env = env_for(name, "f32", R, C, seed=77)
    ref = oracle_outputs(name, env)
    h = fx.fx_expr_create(name, STORAGE_CODE["f32"])
    try:
        n_in, n_out, _, kind = fx.fx_expr_info(h)
        keep = []
        for k, s in enumerate(SLOTS[name]):
            b = env[s]
            t = to_device(b)
            keep.append(t)
            fx.fx_expr_bind(h, k, t.data_ptr(), b.rows, b.cols, b.ld)
        outs = {}
        if kind in ("elementwise", "multi"):
            z = canary_buffer(R * C, torch.float32)
            fx.fx_expr_bind(h, n_in, z.data_ptr(), R, C, R)
            outs["Z"] = z
        if kind in ("full_reduce", "multi"):
            s = canary_buffer(1, torch.float32)
            fx.fx_expr_bind(h, n_in + (1 if kind == "multi" else 0), s.data_ptr(), 1, 1, 1)
            outs["s"] = s
        if kind == "dim_reduce":
            nv = C if name == "schur_colsum" else R
            v = canary_buffer(nv, torch.float32)
            if name == "schur_colsum":
                fx.fx_expr_bind(h, n_in, v.data_ptr(), 1, C, 1)
            else:
                fx.fx_expr_bind(h, n_in, v.data_ptr(), R, 1, R)
            outs["v"] = v
        steps = [("fused", (256, 4, 0, 0)), ("unfused", None), ("fused", (256, 4, 0, 0)),
                 ("fused", (64, 2, 1, 2)), ("fused", (512, 8, 0, 1)), ("unfused", None),
                 ("fused", (128, 2, 2, 0))]
        for i, (how, shape) in enumerate(steps):
            for t in outs.values():
                t.fill_(float("nan"))
            if shape:
                fx.fx_expr_set_launch_shape(h, *shape)
                fx.fx_eval(h, 0)
            else:
                fx.fx_eval_unfused(h, 0)
            torch.cuda.synchronize()
            fx.fx_expr_sync_status(h, 0)
            got = {}
            for key, t in outs.items():
                if key == "Z":
                    got["Z"] = from_device(t[:R * C], "f32").reshape(C, R).T
                elif key == "s":
                    got["s"] = from_device(t[:1], "f64")[0]
                else:
                    got["v"] = from_device(t[:len(t) - 64], "f64")
            check(name, "f32", got, ref, f" step {i} ({how}, {shape})")
    finally:
        fx.fx_expr_destroy(h)
