"""fx_eval_host: inputs copied up from pinned host memory, the tree
evaluated, outputs copied back (GPU).

Element-wise trees whose inputs are each read in one mode run as a
pipeline of column chunks over two internal copy streams; the others
(reductions, multi-output trees, trees that read one input both plainly and
transposed) copy, evaluate and copy back in order. Both are checked against
the FP64 oracle, with device leading dimensions above the row count (pitched
copies), ragged last chunks, explicit streams and the default stream.
"""
import numpy as np
import pytest

import synth
from harness import (SLOTS, STORAGE_CODE, from_device, oracle_outputs, scaled_error, specs_for,
                     tolerance, torch_dtype)

pytestmark = pytest.mark.gpu

DIST = {"schur_exp_trans": "uniform", "sqdiff_accu": "uniform", "schur_trans_accu": "uniform",
        "sigmoid_sqloss": "normal_half"}


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


def _pinned(buf):
    """Dense pinned host copy of a synth buffer (ld = rows)."""
    import torch
    assert buf.ld == max(buf.rows, 1)
    data = np.ascontiguousarray(buf.data[: buf.rows * buf.cols])
    if buf.storage == "bf16":
        t = torch.from_numpy(data.view(np.int16).copy()).view(torch.bfloat16)
    else:
        t = torch.from_numpy(data.copy())
    return t.pin_memory()


def host_run(fx, name, storage, env, R, C, pad=0, explicit_stream=True):
    """fx_eval_host with device buffers of leading dimension rows + pad."""
    import torch
    h = fx.fx_expr_create(name, STORAGE_CODE[storage])
    try:
        n_in, n_out, _, kind = fx.fx_expr_info(h)
        keep, host_in = [], []
        tdt = torch_dtype(storage)
        for k, s in enumerate(SLOTS[name]):
            b = env[s]
            ld = b.rows + pad
            d = torch.full((ld * b.cols + 8,), float("nan"), dtype=tdt, device="cuda")
            keep.append(d)
            fx.fx_expr_bind(h, k, d.data_ptr(), b.rows, b.cols, ld)
            hp = _pinned(b)
            keep.append(hp)
            host_in.append(hp.data_ptr())
        outs, host_out = {}, []
        rdt = torch.float64 if storage == "f64" else torch.float32
        if kind in ("elementwise", "multi"):
            ldz = R + pad
            z = torch.full((ldz * C + 8,), float("nan"), dtype=tdt, device="cuda")
            fx.fx_expr_bind(h, n_in, z.data_ptr(), R, C, ldz)
            hz = torch.full((R * C,), float("nan"), dtype=tdt).pin_memory()
            outs["Z"] = hz
            host_out.append(hz.data_ptr())
            keep.append(z)
        if kind in ("full_reduce", "multi"):
            s = torch.zeros(1, dtype=rdt, device="cuda")
            fx.fx_expr_bind(h, n_in + (1 if kind == "multi" else 0), s.data_ptr(), 1, 1, 1)
            hs = torch.full((1,), float("nan"), dtype=rdt).pin_memory()
            outs["s"] = hs
            host_out.append(hs.data_ptr())
            keep.append(s)
        stream = torch.cuda.Stream() if explicit_stream else None
        sp = int(stream.cuda_stream) if stream is not None else 0
        fx.fx_eval_host(h, host_in, host_out, sp)
        if stream is not None:
            stream.synchronize()
        torch.cuda.synchronize()
        fx.fx_expr_sync_status(h, sp)
        got = {}
        for key, t in outs.items():
            v = from_device(t, storage if key == "Z" else ("f64" if storage == "f64" else "f32"))
            got[key] = v.reshape(C, R).T if key == "Z" else v[0]
        got["_launches"] = fx.fx_expr_last_launches(h)
        return got
    finally:
        fx.fx_expr_destroy(h)


def check(name, storage, got, env, label):
    for key, (rv, rs) in oracle_outputs(name, env).items():
        tol = tolerance(name, storage, key)
        st = storage if key == "Z" else ("f64" if storage == "f64" else "f32")
        err, _, bad, _ = scaled_error(got[key], rv, rs, st)
        assert bad == 0, f"{name}/{storage}/{key}{label}: {bad} wrong non-finite outputs"
        assert err <= tol, f"{name}/{storage}/{key}{label}: scaled error {err:.3e} > {tol:.1e}"


@pytest.mark.parametrize("storage", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("name", ["schur_exp_trans", "schur_sqrt_sigmoid", "add16", "sigmoid"])
def test_pipelined_elementwise(fx, name, storage):
    if name in ("add16", "sigmoid") and storage != "f32":
        pytest.skip("FP32-only tree")
    for k, (R, C, pad) in enumerate([(300, 1000, 0), (257, 129, 8), (64, 40, 0), (97, 31, 4)]):
        env = synth.operands(70 + k, specs_for(name, R, C), storage, DIST.get(name, "normal"))
        for explicit in (True, False):
            got = host_run(fx, name, storage, env, R, C, pad=pad, explicit_stream=explicit)
            check(name, storage, got, env, f" at {R}x{C} pad {pad}")
            if C >= 32:  # one launch per chunk
                assert got["_launches"] > 1


@pytest.mark.parametrize("name", ["sqdiff_accu", "diff_norm", "schur_trans_accu", "expr1"])
def test_in_order_path(fx, name):
    R, C = (200, 200) if name == "expr1" else (300, 170)
    env = synth.operands(80, specs_for(name, R, C), "f32", DIST.get(name, "normal"))
    got = host_run(fx, name, "f32", env, R, C, pad=4)
    check(name, "f32", got, env, f" at {R}x{C}")
    assert got["_launches"] == 1
