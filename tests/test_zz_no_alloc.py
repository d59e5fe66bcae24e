"""fx_sqdiff_accu_f32_noalloc against the FP64 oracle and against fx_eval on
"sqdiff_accu" (GPU).

The no-allocation entry point serves callers that cannot call cudaMalloc
while they compute (a device-memory budget fixed in advance, code that must
not pick up the synchronisation cudaMalloc/cudaFree can cause, or an
allocator owned by another framework). It must give the oracle's sum within
the FP32 reduction tolerance, and the same sum as the ordinary fused
evaluation, on calls in a row that reuse its fixed device scratch array:
dense and strided matrices with 16-byte aligned bases (vector kernels),
bases one float off alignment (single-lane kernels), and an empty matrix,
whose sum is 0. This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from harness import oracle_outputs
from oracle.compare import ErrorReport

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the FP32 reduction tolerance used by the parity tests

# (seed, rows, cols, ld, offset in floats): flat 4-lane, tiled 4-lane,
# flat 1-lane, tiled 1-lane, empty
CASES = [(21, 1000, 700, 1000, 0), (22, 513, 301, 520, 0), (23, 777, 301, 777, 1),
         (24, 300, 211, 303, 1), (25, 0, 40, 1, 0)]


def _entry(fxlib):
    f = ctypes.CDLL(fxlib.lib_path).fx_sqdiff_accu_f32_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return f


def _existing(fxlib, pa, pb, R, C, ld, torch):
    out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    h = fxlib.fx_expr_create("sqdiff_accu", fxlib.FX_F32)
    try:
        fxlib.fx_expr_bind(h, 0, pa, R, C, ld)
        fxlib.fx_expr_bind(h, 1, pb, R, C, ld)
        fxlib.fx_expr_bind(h, 2, out.data_ptr(), 1, 1, 1)
        fxlib.fx_eval(h, 0)
        torch.cuda.synchronize()
    finally:
        fxlib.fx_expr_destroy(h)
    return float(out.item())


def _device(buf, off, torch):
    t = torch.zeros(buf.data.size + off + 4, dtype=torch.float32, device="cuda")
    t[off:off + buf.data.size] = torch.from_numpy(buf.data).cuda()
    return t, t.data_ptr() + 4 * off


def test_noalloc_matches_oracle_and_fx_eval_on_calls_in_a_row(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = _entry(fxlib)
    for seed, R, C, ld, off in CASES:
        env = synth.operands(seed, [("A", R, C), ("B", R, C)], "f32", "uniform",
                             lds={"A": ld, "B": ld})
        A, pa = _device(env["A"], off, torch)
        B, pb = _device(env["B"], off, torch)
        s = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        status = f(pa, pb, R, C, ld, s.data_ptr(), None)
        assert status == 0, fxlib.fx_last_error_string()
        torch.cuda.synchronize()
        got = float(s.item())
        v, m = oracle_outputs("sqdiff_accu", env)["s"]
        rep = ErrorReport("f32", TOL, "m").add([got], [v], mag=[m])
        assert rep.nonfinite == 0 and rep.err <= TOL, (R, C, ld, off, got, v, rep.err)
        want = _existing(fxlib, pa, pb, R, C, ld, torch)
        assert abs(got - want) <= TOL * max(abs(want), m), (R, C, ld, off, got, want)
        if R * C == 0:
            assert got == 0.0


def test_noalloc_refuses_bad_arguments(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = _entry(fxlib)
    s = torch.zeros(1, dtype=torch.float32, device="cuda")
    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = a.data_ptr()
    assert f(p, p, 4, 4, 4, None, None) != 0                 # no output
    assert f(p, p, -1, 4, 4, s.data_ptr(), None) != 0        # negative shape
    assert f(p, p, 4, 4, 3, s.data_ptr(), None) != 0         # ld < rows
    assert f(p + 2, p, 4, 4, 4, s.data_ptr(), None) != 0     # misaligned
    assert f(p, p, 1 << 40, 1 << 40, 1 << 40, s.data_ptr(), None) != 0   # index overflow
    torch.cuda.synchronize()
    assert np.isfinite(float(s.item()))
