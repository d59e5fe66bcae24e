"""fx_sqdiff_accu_f32_noalloc against fx_eval on "sqdiff_accu" (GPU).

The no-allocation entry point serves callers that cannot call cudaMalloc
while they compute (a device-memory budget fixed in advance, code that must
not pick up the synchronisation cudaMalloc/cudaFree can cause, or an
allocator owned by another framework). It must give the same sum as the
ordinary fused evaluation, and keep doing so on a second call that reuses
its fixed device scratch array. This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the FP32 reduction tolerance used by the parity tests


def _entry(fxlib):
    f = ctypes.CDLL(fxlib.lib_path).fx_sqdiff_accu_f32_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return f


def _existing(fxlib, A, B, R, C, ld, torch):
    out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    h = fxlib.fx_expr_create("sqdiff_accu", fxlib.FX_F32)
    try:
        fxlib.fx_expr_bind(h, 0, A.data_ptr(), R, C, ld)
        fxlib.fx_expr_bind(h, 1, B.data_ptr(), R, C, ld)
        fxlib.fx_expr_bind(h, 2, out.data_ptr(), 1, 1, 1)
        fxlib.fx_eval(h, 0)
        torch.cuda.synchronize()
    finally:
        fxlib.fx_expr_destroy(h)
    return float(out.item())


def test_noalloc_matches_fx_eval_on_two_calls(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = _entry(fxlib)
    # call 1: dense 1000 x 700 (flat kernel); call 2: 513 x 301 with ld 520 (tiled kernel)
    for seed, R, C, ld in [(21, 1000, 700, 1000), (22, 513, 301, 520)]:
        env = synth.operands(seed, [("A", R, C), ("B", R, C)], "f32", "uniform",
                             lds={"A": ld, "B": ld})
        A = torch.from_numpy(env["A"].data).cuda()
        B = torch.from_numpy(env["B"].data).cuda()
        s = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        status = f(A.data_ptr(), B.data_ptr(), R, C, ld, s.data_ptr(), None)
        assert status == 0, fxlib.fx_last_error_string()
        torch.cuda.synchronize()
        got = float(s.item())
        want = _existing(fxlib, A, B, R, C, ld, torch)
        assert abs(got - want) <= TOL * abs(want), (R, C, got, want)
