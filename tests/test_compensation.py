"""The compensated FP32 reductions on the GPU, on sums where compensation
decides the answer (GPU).

Each case is built so that the exact sum is known in closed form and a
plain FP32 accumulation, taken in the kernel's own order (per-thread
running sums over the kernel's vectors and unrolled steps, then the warp
and block butterflies), visibly misses it. The kernel must stay within a
few FP32 ulps of the exact value; the test computes, on the host in numpy
float32, what the plain accumulation would have returned and asserts that
it breaks the same bound, so the pass is owed to the compensation.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

F = np.float32
ULPS = 4          # the bound: |result - exact| <= 4 ulps of the exact value in FP32


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


def _pairwise(vals):
    """The kernels' lane sum: adjacent pairs first, in FP32."""
    vals = [F(v) for v in vals]
    while len(vals) > 1:
        vals = [F(vals[2 * j] + vals[2 * j + 1]) for j in range(len(vals) // 2)]
    return vals[0]


def _butterfly(x):
    """xor-shuffle butterfly over the last axis (32 lanes), plain FP32 adds."""
    for o in (16, 8, 4, 2, 1):
        x = (x + x[..., np.arange(32) ^ o]).astype(F)
    return x[..., 0]


def plain_flat_accu(n, V, U, block, grid, t):
    """What the flat reduction kernel would return for n equal terms t if
    every FP32 add were plain: thread g of the grid takes, in step k, the
    vectors b_g + k*step + u*block (u < U) that exist, sums each vector's V
    lanes and then the U vector sums pairwise, and adds that to its running
    sum; warps and blocks combine by butterflies; block partials are summed
    in FP64 (as the kernel does)."""
    nv = n // V
    T = grid * block
    g = np.arange(T)
    b = (g // block) * block * U + g % block
    step = grid * block * U
    vt = _pairwise([t] * V)
    table = np.array([_pairwise([vt] * c + [F(0)] * (U - c)) for c in range(U + 1)], dtype=F)
    s = np.zeros(T, dtype=F)
    k = 0
    while np.any(b + k * step < nv):
        base = b + k * step
        cnt = sum((base + u * block < nv).astype(np.int64) for u in range(U))
        act = cnt > 0
        s[act] = (s[act] + table[cnt[act]]).astype(F)
        k += 1
    w = _butterfly(s.reshape(grid, block // 32, 32))
    lanes = np.zeros((grid, 32), dtype=F)
    lanes[:, : block // 32] = w
    return F(math.fsum(_butterfly(lanes).astype(np.float64).tolist()))


def ulps_off(got, exact):
    return abs(float(got) - exact) / float(np.spacing(F(exact)))


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _sqdiff_accu(fx, storage, A, B, R, C, shape):
    import torch
    code = {"f32": fx.FX_F32, "bf16": fx.FX_BF16}[storage]
    out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    h = fx.fx_expr_create("sqdiff_accu", code)
    try:
        fx.fx_expr_set_launch_shape(h, *shape)
        fx.fx_expr_bind(h, 0, A.data_ptr(), R, C, R)
        fx.fx_expr_bind(h, 1, B.data_ptr(), R, C, R)
        fx.fx_expr_bind(h, 2, out.data_ptr(), 1, 1, 1)
        fx.fx_eval(h, 0)
        torch.cuda.synchronize()
        fx.fx_expr_sync_status(h, 0)
    finally:
        fx.fx_expr_destroy(h)
    return F(out.item())


@pytest.mark.parametrize("storage,size,a,b,vec,unroll", [
    # fl32(sqrt(0.1))^2 = 0.1 in FP32, 8192^2 terms, 4 lanes per vector, 2 vectors a step
    ("f32", 8192, math.sqrt(0.1), 0.0, 4, 2),
    # bf16(0.1) - bf16(-2^-12): a 24-bit square, 16384^2 terms, 8 lanes, 4 vectors a step
    ("bf16", 16384, 0.1, -2.0 ** -12, 8, 4)])
def test_long_sum_of_equal_terms(fx, storage, size, a, b, vec, unroll):
    import torch
    R = C = size
    n = R * C
    av, bv = (synth.to_f64(synth.round_to_storage(np.array([x]), storage), storage)[0]
              for x in (a, b))
    d = F(F(av) - F(bv))
    t = F(d * d)                                 # the term, as the kernel computes it in FP32
    exact = n * float(t)                         # exact in FP64 (t has 24 bits, n = 2^26 / 2^28)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    A = torch.full((n,), float(av), dtype=dt, device="cuda")
    B = torch.full((n,), float(bv), dtype=dt, device="cuda")
    # register-load kernel, one block per SM: long per-thread chains
    shape = (256, unroll, 1, 2)
    got = _sqdiff_accu(fx, storage, A, B, R, C, shape)
    plain = plain_flat_accu(n, vec, unroll, 256, min(_sms(), n // vec // (256 * unroll) + 1), t)
    e_got, e_plain = ulps_off(got, exact), ulps_off(plain, exact)
    print(f"accu of {n} x {float(t)!r} ({storage}): kernel {e_got:.1f} ulps, "
          f"plain FP32 in the kernel's order {e_plain:.1f} ulps")
    assert e_plain > ULPS, "the case does not separate compensated from plain sums"
    assert e_got <= ULPS, f"kernel result {float(got)!r} is {e_got:.1f} ulps from {exact!r}"


def test_cancelling_column_sums(fx):
    """sum(X % Y, 0) with Y = 1 and, in every column, rows whose thread
    lane (row / 4 mod 256 for 4-lane FP32 vectors) is below 16 within its
    warp holding s, and the other lanes alternating +L and -L. Each thread's
    32 elements are equal, so its own sum is exact; in the butterfly a
    plain FP32 add meets 32s against 32L (below half an ulp) before the +L
    and -L cancel, and the s terms vanish. The exact sum is 4096 s per
    8192 rows."""
    import torch
    R, C = 8192, 64
    L, s_small = 2.0 ** 20, 2.0 ** -5
    rows = np.arange(R)
    lane = (rows // 4) % 256
    wl = lane % 32
    col = np.where(wl < 16, s_small, np.where(wl % 2 == 0, L, -L))
    scale = 1.0 + np.arange(C) / 8.0           # vary the columns (exact in FP32)
    X = (col[:, None] * scale[None, :]).astype(np.float32)
    exact = np.array([4096 * s_small * sc for sc in scale])
    Xd = torch.from_numpy(np.asfortranarray(X).ravel(order="F")).cuda()
    Yd = torch.ones(R * C, dtype=torch.float32, device="cuda")
    out = torch.full((C,), float("nan"), dtype=torch.float32, device="cuda")
    h = fx.fx_expr_create("schur_colsum", fx.FX_F32)
    try:
        fx.fx_expr_bind(h, 0, Xd.data_ptr(), R, C, R)
        fx.fx_expr_bind(h, 1, Yd.data_ptr(), R, C, R)
        fx.fx_expr_bind(h, 2, out.data_ptr(), 1, C, 1)
        fx.fx_eval(h, 0)
        torch.cuda.synchronize()
        fx.fx_expr_sync_status(h, 0)
    finally:
        fx.fx_expr_destroy(h)
    got = out.cpu().numpy().astype(np.float64)
    # plain FP32 in the kernel's order: per thread the 32 equal elements
    # (exact), then the block butterflies of warp totals
    plain = []
    for j in range(C):
        thr = (32 * X[::4, j][:256]).astype(F)          # one value per thread (lane 0..255)
        w = _butterfly(thr.reshape(8, 32))
        lanes = np.zeros(32, dtype=F)
        lanes[:8] = w
        plain.append(float(_butterfly(lanes[None, :])[0]))
    plain = np.array(plain)
    e_got = np.abs(got - exact) / np.spacing(exact.astype(F)).astype(np.float64)
    e_plain = np.abs(plain - exact) / np.spacing(exact.astype(F)).astype(np.float64)
    print(f"cancelling colsum: kernel max {e_got.max():.1f} ulps, plain FP32 min "
          f"{e_plain.min():.3g} ulps")
    assert np.all(e_plain > ULPS)
    assert np.all(e_got <= ULPS), (got[:4], exact[:4])
