"""The C ABI library loads, exports every declared entry point, and checks
its arguments on the host (no GPU needed: none of these calls reach CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

EXPECTED = {
    "schur_exp_trans": (4, 1, 1, "elementwise"),
    "sqdiff_accu": (2, 1, 0, "full_reduce"),
    "schur_sqrt_sigmoid": (4, 1, 1, "elementwise"),
    "schur_colsum": (2, 1, 0, "dim_reduce"),
    "absdiff_rowmax": (2, 1, 0, "dim_reduce"),
    "diff_norm": (2, 1, 0, "full_reduce"),
    "schur_trans_accu": (3, 2, 1, "multi"),
    "sigmoid_sqloss": (4, 1, 0, "full_reduce"),
}


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fx_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(fxlib):
    names = declared_functions()
    assert len(names) >= 19
    L = ctypes.CDLL(fxlib.lib_path)
    for n in names:
        assert hasattr(L, n), n


def test_registry_lists_expected_trees(fxlib):
    listed = {(n, d) for n, d, _ in fxlib.fx_list()}
    for name in EXPECTED:
        for d in (fxlib.FX_F32, fxlib.FX_F64, fxlib.FX_BF16, fxlib.FX_F16):
            assert (name, d) in listed, (name, d)


@pytest.mark.parametrize("name", sorted(EXPECTED))
def test_info_and_slots(fxlib, name):
    h = fxlib.fx_expr_create(name, fxlib.FX_F32)
    try:
        assert fxlib.fx_expr_info(h) == EXPECTED[name]
        n_in, n_out = EXPECTED[name][:2]
        names = [fxlib.fx_expr_slot_name(h, k) for k in range(n_in + n_out)]
        assert len(set(names)) == n_in + n_out
        with pytest.raises(fxlib.FxError):
            fxlib.fx_expr_slot_name(h, n_in + n_out)
    finally:
        fxlib.fx_expr_destroy(h)


def test_create_errors(fxlib):
    with pytest.raises(fxlib.FxError) as e:
        fxlib.fx_expr_create("no_such_tree", fxlib.FX_F32)
    assert e.value.status == -9
    with pytest.raises(fxlib.FxError) as e:
        fxlib.fx_expr_create("schur_exp_trans", 7)
    assert e.value.status == -1


def test_bind_checks(fxlib):
    h = fxlib.fx_expr_create("schur_exp_trans", fxlib.FX_F32)
    try:
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_expr_bind(h, 9, 0x1000, 4, 4, 4)
        assert e.value.status == -1
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_expr_bind(h, 0, 0x1000, 8, 4, 4)          # ld < rows
        assert e.value.status == -1
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_expr_bind(h, 0, 0x1002, 4, 4, 4)          # not 4-byte aligned
        assert e.value.status == -4
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_expr_bind(h, 0, 0, 4, 4, 4)               # null, non-empty
        assert e.value.status == -1
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_expr_bind(h, 0, 0x1000, -1, 4, 4)
        assert e.value.status == -2
        fxlib.fx_expr_bind(h, 0, 0, 0, 0, 1)                   # empty is fine
    finally:
        fxlib.fx_expr_destroy(h)


def test_unbound_and_shape_errors_before_any_launch(fxlib):
    h = fxlib.fx_expr_create("schur_exp_trans", fxlib.FX_F32)
    try:
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_eval(h)
        assert e.value.status == -5
        for k in range(3):
            fxlib.fx_expr_bind(h, k, 0x1000, 8, 6, 8)
        fxlib.fx_expr_bind(h, 3, 0x1000, 8, 6, 8)            # D must be 6 x 8
        fxlib.fx_expr_bind(h, 4, 0x1000, 8, 6, 8)
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_eval(h)
        assert e.value.status == -2
        assert "slot 3" in fxlib.fx_last_error_string()
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_eval_backward(h, 0, [0] * 4)
        assert e.value.status == -6
    finally:
        fxlib.fx_expr_destroy(h)


def test_reduction_output_shape_checked(fxlib):
    h = fxlib.fx_expr_create("schur_colsum", fxlib.FX_F64)
    try:
        fxlib.fx_expr_bind(h, 0, 0x1000, 8, 6, 8)
        fxlib.fx_expr_bind(h, 1, 0x1000, 8, 6, 8)
        fxlib.fx_expr_bind(h, 2, 0x1000, 8, 1, 8)            # colsum is 1 x 6
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_eval(h)
        assert e.value.status == -2
    finally:
        fxlib.fx_expr_destroy(h)


def test_scalars(fxlib):
    h = fxlib.fx_expr_create("schur_exp_trans", fxlib.FX_BF16)
    try:
        assert fxlib.fx_expr_get_scalar(h, 0) == 3.5
        fxlib.fx_expr_set_scalar(h, 0, -1.25)
        assert fxlib.fx_expr_get_scalar(h, 0) == -1.25
        with pytest.raises(fxlib.FxError):
            fxlib.fx_expr_set_scalar(h, 1, 0.0)
    finally:
        fxlib.fx_expr_destroy(h)


def test_status_strings(fxlib):
    for s in range(0, -10, -1):
        assert fxlib.fx_status_string(s)
    fxlib.fx_expr_destroy(None)


def test_slot_dtypes(fxlib):
    h = fxlib.fx_expr_create("expr3", fxlib.FX_F32)
    try:
        assert [fxlib.fx_expr_slot_dtype(h, k) for k in range(4)] == [
            fxlib.FX_F32, fxlib.FX_F64, fxlib.FX_F32, fxlib.FX_F32]
        # the FP64 slot wants 8-byte alignment
        with pytest.raises(fxlib.FxError) as e:
            fxlib.fx_expr_bind(h, 1, 0x1004, 8, 6, 8)
        assert e.value.status == -4
        fxlib.fx_expr_bind(h, 0, 0x1004, 8, 6, 8)
    finally:
        fxlib.fx_expr_destroy(h)
    h = fxlib.fx_expr_create("sqdiff_accu", fxlib.FX_BF16)
    try:
        assert fxlib.fx_expr_slot_dtype(h, 0) == fxlib.FX_BF16
        assert fxlib.fx_expr_slot_dtype(h, 2) == fxlib.FX_F32      # the accu output
        with pytest.raises(fxlib.FxError):
            fxlib.fx_expr_slot_dtype(h, 3)
    finally:
        fxlib.fx_expr_destroy(h)


def test_product_trees_listed(fxlib):
    h = fxlib.fx_expr_create("gemm_scale", fxlib.FX_BF16)
    try:
        assert fxlib.fx_expr_info(h)[:2] == (2, 1)
    finally:
        fxlib.fx_expr_destroy(h)
    h = fxlib.fx_expr_create("chain", fxlib.FX_F32)
    fxlib.fx_expr_destroy(h)


def test_launch_shape_validation(fxlib):
    """fx_expr_set_launch_shape accepts the documented ranges (block 64-512
    in warps, unroll 2/4/8, blocks per SM 0-32, pipeline 0-2), rejects the rest
    without changing the shape in force, and reads back what it set."""
    h = fxlib.fx_expr_create("schur_sqrt_sigmoid", fxlib.FX_F32)
    try:
        assert fxlib.fx_expr_launch_shape(h) == (256, 4, 0, 0)
        for good in [(64, 2, 0, 0), (512, 8, 32, 2), (96, 4, 1, 1), (256, 2, 4, 2)]:
            fxlib.fx_expr_set_launch_shape(h, *good)
            assert fxlib.fx_expr_launch_shape(h) == good
        before = fxlib.fx_expr_launch_shape(h)
        for bad in [(48, 4, 0, 0), (100, 4, 0, 0), (544, 4, 0, 0), (256, 1, 0, 0), (256, 3, 0, 0),
                    (256, 16, 0, 0), (256, 4, -1, 0), (256, 4, 33, 0), (256, 4, 0, -1),
                    (256, 4, 0, 3)]:
            with pytest.raises(fxlib.FxError):
                fxlib.fx_expr_set_launch_shape(h, *bad)
            assert fxlib.fx_expr_launch_shape(h) == before
    finally:
        fxlib.fx_expr_destroy(h)


def test_batch_rejects_operands_beyond_32bit_offsets(fxlib):
    """fx_eval_batch refuses, on the host and before any launch, items whose
    matrix operands span 2^31 elements or more (the batched kernel's 32-bit
    offsets); the pointers are never dereferenced."""
    FX_E_SHAPE = -2
    h = fxlib.fx_expr_create("schur_trans_accu", fxlib.FX_F32)   # A, B, C (transposed), Z, s
    try:
        def item(R, C, ld=None):
            it = (fxlib.BatchItem * 1)()
            for k in range(5):
                it[0].ptr[k] = 0x10000000 + k * 0x1000000
            for k, v in (ld or {}).items():
                it[0].ld[k] = v
            it[0].rows, it[0].cols = R, C
            return it
        cases = [item(1 << 16, 1 << 16),                 # 2^32 elements
                 item(1000, 1000, {0: 1 << 22}),         # A's leading dimension
                 item(1000, 1000, {2: 1 << 22}),         # the transposed C (cols x rows)
                 item(1000, 1000, {3: 1 << 22}),         # Z
                 item(1 << 31, 1)]                       # rows beyond int32
        for it in cases:
            with pytest.raises(fxlib.FxError) as e:
                fxlib.fx_eval_batch(h, it, 0, True)
            assert e.value.status == FX_E_SHAPE, fxlib.fx_last_error_string()
    finally:
        fxlib.fx_expr_destroy(h)
