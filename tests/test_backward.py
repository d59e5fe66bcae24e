"""Fused backward of L = accu(square(sigmoid(X % W + b.each_col) - Y)) (GPU):
gradients against the oracle's reverse pass (with its error bound) and
against finite differences; the torch.autograd.Function wrapper."""
import math

import numpy as np
import pytest

import oracle
import synth
from harness import STORAGE_CODE, from_device, run, scaled_error, to_device, torch_dtype
from oracle import grad as ograd

pytestmark = pytest.mark.gpu

LOSS = "(accu (square (- (sigmoid (+ (% X W) (each_col b))) Y)))"
SLOTS = "XWYb"
TOL = {"f64": 1e-13, "f32": 1e-5, "bf16": 8e-3, "f16": 1e-3}


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


def env_for(storage, R, C, seed=3):
    return synth.operands(seed, [("X", R, C), ("W", R, C), ("Y", R, C), ("b", R, 1)], storage,
                          "normal_half")


def gpu_grads(fx, storage, env, want=SLOTS, gL=None):
    """dL/d(slot) for the slots in `want` via fx_eval_backward (dense outputs)."""
    import torch
    dev = {s: to_device(env[s]) for s in SLOTS}
    h = fx.fx_expr_create("sigmoid_sqloss", STORAGE_CODE[storage])
    try:
        for k, s in enumerate(SLOTS):
            b = env[s]
            fx.fx_expr_bind(h, k, dev[s].data_ptr(), b.rows, b.cols, b.ld)
        grads = {}
        for s in want:
            b = env[s]
            t = torch.empty(b.rows * b.cols + 64, dtype=torch_dtype(storage), device="cuda")
            t.fill_(float("nan"))
            grads[s] = t
        ptrs = [grads[s].data_ptr() if s in grads else 0 for s in SLOTS]
        g_dev = None
        if gL is not None:
            g_dev = torch.tensor([gL], dtype=torch.float64 if storage == "f64" else torch.float32,
                                 device="cuda")
        fx.fx_eval_backward(h, g_dev.data_ptr() if g_dev is not None else 0, ptrs)
        torch.cuda.synchronize()
        fx.fx_expr_sync_status(h, 0)
        launches = fx.fx_expr_last_launches(h)
    finally:
        fx.fx_expr_destroy(h)
    out = {}
    for s, t in grads.items():
        b = env[s]
        n = b.rows * b.cols
        assert bool(torch.isnan(t[n:].float()).all()), f"d{s}: write past the end"
        out[s] = from_device(t[:n], storage)       # dense column-major, flat
    return out, launches


def check_grads(got, ref, storage, label):
    for s, (idx, v, sg) in ref.items():
        if s not in got:
            continue
        g = got[s][idx]
        err, _, bad, _ = scaled_error(g, v, sg, storage)
        assert bad == 0, f"d{s} {label}: non-finite"
        assert err <= TOL[storage], f"d{s} {label}: scaled error {err:.3e} > {TOL[storage]}"


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_gradients_small(fx, storage):
    for R, C in [(1, 1), (7, 5), (64, 48), (100, 37), (257, 129)]:
        env = env_for(storage, R, C)
        for gL in (None, 0.75):
            got, launches = gpu_grads(fx, storage, env, gL=gL)
            ref = ograd.gradient_sigma(LOSS, env, 1.0 if gL is None else gL)
            check_grads(got, ref, storage, f"at {R}x{C}, gL={gL}")
            assert launches == 1


def test_partial_request_writes_only_requested(fx):
    env = env_for("f32", 96, 80)
    got, _ = gpu_grads(fx, "f32", env, want="Xb")
    assert set(got) == {"X", "b"}
    ref = ograd.gradient_sigma(LOSS, env)
    check_grads(got, ref, "f32", "(X and b only)")


def test_zero_weights_closed_form(fx):
    env = env_for("f32", 64, 32)
    env["W"].data[:] = 0
    got, _ = gpu_grads(fx, "f32", env, want="X")
    assert np.all(got["X"] == 0.0)


def test_backward_repeatable(fx):
    env = env_for("f32", 700, 600)
    a, _ = gpu_grads(fx, "f32", env)
    b, _ = gpu_grads(fx, "f32", env)
    for s in a:
        assert np.array_equal(a[s], b[s]), s


def gradient_reports(got, env, storage, block=128):
    """Every element of every gradient against the oracle's reverse pass:
    the output rows in blocks of `block` (a row block of X, W, Y is read only
    by those output rows, and b(i) only by row i, so each block's gradient
    entries are exact), evaluated on a thread pool."""
    from concurrent.futures import ThreadPoolExecutor

    from harness import _workers
    from oracle.compare import ErrorReport
    R = env["X"].rows

    def one(r0):
        ref = ograd.gradient_sigma(LOSS, env, 1.0, rows=np.arange(r0, min(R, r0 + block)))
        out = {}
        for s_, (idx, v, sg) in ref.items():
            if s_ in got:
                out[s_] = ErrorReport(storage, TOL[storage], "sigma").add(got[s_][idx], v, sg)
        return out

    total = {}
    with ThreadPoolExecutor(_workers()) as ex:
        for part in ex.map(one, range(0, R, block)):
            for s_, rep in part.items():
                if s_ in total:
                    total[s_].merge(rep)
                else:
                    total[s_] = rep
    return total


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_gradients_8192_all_elements_and_finite_differences(fx, storage):
    from harness import record
    R = C = 8192
    env = env_for(storage, R, C)
    got, _ = gpu_grads(fx, storage, env)
    reps = gradient_reports(got, env, storage)
    for s_, rep in reps.items():
        record(f"sigmoid_sqloss/{storage}/d{s_} at 8192^2", rep)
        assert rep.nonfinite == 0, f"d{s_}: non-finite"
        assert rep.err <= TOL[storage], f"d{s_} at 8192^2: scaled error {rep.err:.3e}"
        assert rep.n == (R if s_ == "b" else R * C)
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(R, 64, replace=False))
    # finite differences: L is a sum of per-element terms, so perturbing X(i,j)
    # or W(i,j) changes term (i,j) only, and b(i) changes row i only
    f64 = {s: env[s].f64() for s in SLOTS}
    for k in range(64):
        i, j = int(rng.integers(R)), int(rng.integers(C))
        x, w, y, bb = (f64["X"][i + j * R], f64["W"][i + j * R], f64["Y"][i + j * R], f64["b"][i])

        def term(x_, w_, b_):
            return (1.0 / (1.0 + math.exp(-(x_ * w_ + b_))) - y) ** 2

        for s, fn, x0 in (("X", lambda v: term(v, w, bb), x), ("W", lambda v: term(x, v, bb), w)):
            h = 1e-6 * max(1.0, abs(x0))
            fd = (fn(x0 + h) - fn(x0 - h)) / (2 * h)
            g = got[s][i + j * R]
            assert abs(g - fd) <= 1e-6 + 1e-4 * abs(fd) + (8e-3 * abs(fd) if storage == "bf16" else 0), (s, i, j, g, fd)
    for i in rows[:8]:
        i = int(i)
        xs, ws, ys = (f64[s][i::R][:C] for s in "XWY")

        def row_loss(b_):
            return float(np.sum((1.0 / (1.0 + np.exp(-(xs * ws + b_))) - ys) ** 2))

        h = 1e-6 * max(1.0, abs(f64["b"][i]))
        fd = (row_loss(f64["b"][i] + h) - row_loss(f64["b"][i] - h)) / (2 * h)
        g = got["b"][i]
        assert abs(g - fd) <= 1e-5 * max(1.0, abs(fd)) + (8e-3 * abs(fd) if storage == "bf16" else 0), (i, g, fd)


def test_forward_loss_8192(fx):
    R = C = 8192
    for storage in ("f32", "bf16"):
        env = env_for(storage, R, C)
        got = run(fx, "sigmoid_sqloss", storage, env, R, C)
        v, s = oracle.evaluate_sigma(LOSS, env)
        err, _, bad, _ = scaled_error([got["s"]], [v[0, 0]], [s[0, 0]], "f32")
        assert bad == 0 and err <= 1e-5, (storage, err)


def test_autograd_function(fx):
    import torch
    R, C = 200, 150
    env = env_for("f32", R, C)
    ts = {}
    for s in SLOTS:
        b = env[s]
        t = fx.colmajor(b.rows, b.cols, torch.float32) if s != "b" else torch.empty(R, device="cuda")
        if s != "b":
            t.copy_(torch.from_numpy(b.data.reshape(b.cols, b.rows).T.copy()))
        else:
            t.copy_(torch.from_numpy(b.data.copy()))
        ts[s] = t.requires_grad_(True)
    F = fx.FusedLoss()
    L = F.apply("sigmoid_sqloss", fx.FX_F32, ts["X"], ts["W"], ts["Y"], ts["b"])
    (2.5 * L).backward()
    ref = oracle.gradient(LOSS, env, gL=2.5)
    for s in SLOTS:
        g = ts[s].grad.double().cpu().numpy()
        r = ref[s] if s != "b" else ref[s][:, 0]
        scale = np.maximum(np.abs(r), 1e-2 * np.max(np.abs(r)))
        assert np.max(np.abs(g - r) / scale) < 1e-4, s
    Lr = oracle.evaluate(LOSS, env)[0, 0]
    assert abs(L.item() - Lr) <= 1e-5 * abs(Lr)
