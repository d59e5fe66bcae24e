"""Trees with matrix products (GPU): the fusion boundary.

Fig. 1's Z = 2 X Y^T (the scalar folded into the GEMM), a product followed
by a fused element-wise remainder, and Sec. 4's chain Z = A * B * C * D,
against the FP64 oracle (whose product error bound is pinned in
test_oracle.py), plus the unfused baseline and shape errors.
"""
import numpy as np
import pytest

import synth
from harness import oracle_outputs, run, scaled_error, tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


def check(name, storage, got, env, label):
    for key, (rv, rs) in oracle_outputs(name, env).items():
        tol = tolerance(name, storage, key)
        err, _, bad, _ = scaled_error(got[key], rv, rs, storage)
        assert bad == 0, f"{name}/{storage}{label}: {bad} wrong non-finite outputs"
        assert err <= tol, f"{name}/{storage}{label}: scaled error {err:.3e} > {tol:.1e}"


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_gemm_scale(fx, storage):
    for k, (R, C, K) in enumerate([(33, 17, 20), (256, 192, 300), (1000, 700, 512), (1, 1, 1),
                                   (5, 7, 0)]):
        env = synth.operands(90 + k, [("X", R, K), ("Y", C, K)], storage, "uniform")
        got = run(fx, "gemm_scale", storage, env, R, C)
        check("gemm_scale", storage, got, env, f" at {R}x{C}, K={K}")
        # X (R x K) and Y (C x K) are TMA-addressable when their leading
        # dimensions are multiples of 16 bytes
        if storage in ("bf16", "f16") and R * C * K > 0 and (R * 2) % 16 == 0 and (C * 2) % 16 == 0:
            assert got["_launches"] == 1  # the tensor-core kernel (TMA-addressable operands)
        else:
            assert got["_launches"] == 0  # one library GEMM, no fused pass


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_gemm_epilogue(fx, storage):
    for k, (R, C, K) in enumerate([(64, 48, 40), (300, 257, 129), (1024, 512, 256)]):
        env = synth.operands(95 + k, [("X", R, K), ("Y", K, C), ("W", R, C)], storage, "normal")
        got = run(fx, "gemm_epilogue", storage, env, R, C)
        check("gemm_epilogue", storage, got, env, f" at {R}x{C}, K={K}")
        assert got["_launches"] == 1      # the tensor-core kernel, or the pass after the GEMM
        unf = run(fx, "gemm_epilogue", storage, env, R, C, unfused=True)
        check("gemm_epilogue", storage, unf, env, f" unfused at {R}x{C}")
        assert unf["_launches"] >= 3


def test_chain(fx):
    # decreasing sizes, as in Sec. 4
    for k, dims in enumerate([(256, 192, 128, 96, 64), (500, 333, 200, 101, 37)]):
        R, K1, K2, K3, C = dims
        env = synth.operands(99 + k, [("A", R, K1), ("B", K1, K2), ("C", K2, K3), ("D", K3, C)],
                             "f32", "uniform")
        got = run(fx, "chain", "f32", env, R, C)
        check("chain", "f32", got, env, f" {dims}")


def test_product_shape_error(fx):
    env = synth.operands(98, [("X", 40, 30), ("Y", 20, 31)], "f32", "uniform")
    with pytest.raises(fx.FxError):
        run(fx, "gemm_scale", "f32", env, 40, 20)


# ---------------------------------------------------------------- tensor cores
#
# BF16/FP16 trees with one product run on the tcgen05 kernel (launch-shape
# pipeline 0) when the operands are TMA-addressable; pipelines 1 and 2 take
# the library GEMM and the fused pass. Shapes: whole tiles (128 x 256,
# K in steps of 64), ragged edges in M, N and K, K shorter than one step,
# more K steps than pipeline stages, and sizes from 1024 to 4096.

UMMA_SHAPES = [(128, 256, 64), (256, 512, 512), (200, 300, 72), (1000, 712, 520), (64, 48, 40),
               (1024, 1024, 1024), (2048, 1536, 2048), (4096, 4096, 4096)]


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("name", ["gemm_epilogue", "gemm_scale"])
def test_tensor_core_kernel_against_oracle(fx, name, storage):
    for k, (R, C, K) in enumerate(UMMA_SHAPES):
        if name == "gemm_epilogue":
            specs = [("X", R, K), ("Y", K, C), ("W", R, C)]
        else:
            specs = [("X", R, K), ("Y", C, K)]
        env = synth.operands(120 + k, specs, storage, "normal")
        got = run(fx, name, storage, env, R, C, shape=(256, 4, 0, 0))
        check(name, storage, got, env, f" at {R}x{C}, K={K} (tcgen05)")
        # operands TMA can address: leading dimensions of 16-byte multiples
        lds = [R, K] if name == "gemm_epilogue" else [R, C]
        if all(ld * 2 % 16 == 0 for ld in lds):
            assert got["_launches"] == 1
        else:   # the library GEMM (and, for gemm_epilogue, the fused pass)
            assert got["_launches"] == (1 if name == "gemm_epilogue" else 0)
        lib = run(fx, name, storage, env, R, C, shape=(256, 4, 0, 2))
        check(name, storage, lib, env, f" at {R}x{C}, K={K} (library GEMM)")
