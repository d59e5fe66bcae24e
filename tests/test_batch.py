"""Batched evaluation of Z = A % B + 0.5 * trans(C) and s = accu(Z) over
many matrices of uneven shapes in one persistent launch (GPU)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


def arena(mats, dtype, align=4):
    """One device buffer holding every matrix, each starting `align` elements aligned."""
    import torch
    offs, pos = [], 0
    for m in mats:
        offs.append(pos)
        pos += (m.data.size + align - 1) // align * align
    host = np.zeros(max(pos, 1), dtype=mats[0].data.dtype if mats else np.float32)
    for m, o in zip(mats, offs):
        host[o:o + m.data.size] = m.data
    return torch.from_numpy(host).cuda(), offs


def run_batch(fx, rows, cols, ops, use_graph, repeat=1, storage=0, shape=None, tune=None,
              shape_out=None):
    import torch
    n = len(rows)
    A, oa = arena(ops["A"], None)
    B, ob = arena(ops["B"], None)
    C, oc = arena(ops["C"], None)
    zsizes = [synth.Buffer(np.zeros(r * c, np.float32), r, c, max(r, 1), "f32")
              for r, c in zip(rows, cols)]
    Z, oz = arena(zsizes, None)
    Z.fill_(float("nan"))
    S = torch.full((n,), float("nan"), device="cuda")
    items = (fx.BatchItem * n)()
    es = A.element_size()
    for i in range(n):
        it = items[i]
        it.ptr[0] = A.data_ptr() + oa[i] * es
        it.ptr[1] = B.data_ptr() + ob[i] * es
        it.ptr[2] = C.data_ptr() + oc[i] * es
        it.ptr[3] = Z.data_ptr() + oz[i] * es
        it.ptr[4] = S.data_ptr() + i * 4
        it.rows, it.cols = int(rows[i]), int(cols[i])
    h = fx.fx_expr_create("schur_trans_accu", storage)
    stream = torch.cuda.Stream()
    try:
        if shape is not None:
            fx.fx_expr_set_launch_shape(h, *shape)
        if tune is not None:
            fx.fx_tune_batch(h, items, tune, int(stream.cuda_stream))
        if shape_out is not None:
            shape_out.append(tuple(fx.fx_expr_launch_shape(h)))
        for _ in range(repeat):
            fx.fx_eval_batch(h, items, int(stream.cuda_stream), use_graph)
        stream.synchronize()
        launches = fx.fx_expr_last_launches(h)
    finally:
        fx.fx_expr_destroy(h)
    zs = []
    Zh = Z.cpu().numpy()
    for i in range(n):
        r, c = int(rows[i]), int(cols[i])
        zs.append(Zh[oz[i]:oz[i] + r * c].reshape(c, r).T.astype(np.float64) if r * c else
                  np.zeros((r, c)))
    return zs, S.cpu().numpy().astype(np.float64), launches


def check(ops, rows, cols, zs, ss, which, report=None):
    """Every listed matrix's Z and s against the oracle (gate scale of the
    tree), on a thread pool; with `report` = (label, ...) the summary is
    recorded for the end-of-run error table."""
    from concurrent.futures import ThreadPoolExecutor

    from harness import _workers, oracle_outputs, record
    from oracle.compare import ErrorReport

    def one(i):
        env = {k: ops[k][i] for k in "ABC"}
        ref = oracle_outputs("schur_trans_accu", env)
        z, sz = ref["Z"]
        rz = ErrorReport("f32", 2e-6, "m").add(zs[i], z, mag=sz)
        v, sv = ref["s"]
        rs = ErrorReport("f32", 1e-5, "m").add([ss[i]], [v], mag=[sv])
        assert rz.nonfinite == 0 and rz.err <= 2e-6, (i, rows[i], cols[i], rz.err)
        assert rs.nonfinite == 0 and rs.err <= 1e-5, (i, "s", rs.err)
        return rz, rs

    tz, ts = ErrorReport("f32", 2e-6, "m"), ErrorReport("f32", 1e-5, "m")
    with ThreadPoolExecutor(_workers()) as ex:
        for rz, rs in ex.map(one, list(which)):
            tz.merge(rz)
            ts.merge(rs)
    if report:
        record(f"{report} Z", tz)
        record(f"{report} s", ts)


@pytest.mark.parametrize("use_graph", [False, True])
def test_small_uneven_batch(fx, use_graph):
    rows, cols, ops = synth.batch_operands(5, 60, [("A", False), ("B", False), ("C", True)],
                                           lo=1, hi=300)
    zs, ss, launches = run_batch(fx, rows, cols, ops, use_graph, repeat=2)
    check(ops, rows, cols, zs, ss, range(len(rows)))
    assert launches == 2


def test_graph_replay_matches_direct(fx):
    rows, cols, ops = synth.batch_operands(6, 40, [("A", False), ("B", False), ("C", True)],
                                           lo=8, hi=200)
    z1, s1, _ = run_batch(fx, rows, cols, ops, False)
    z2, s2, _ = run_batch(fx, rows, cols, ops, True, repeat=3)
    assert np.array_equal(s1, s2)
    for a, b in zip(z1, z2):
        assert np.array_equal(a, b)


def test_batch_4096_log_uniform(fx):
    """The batch the benchmark times: 4096 matrices, rows and cols
    log-uniform in [16, 2048] (seed 2), the launch shape autotuned as the
    benchmark does, graph-replayed; every element of every matrix compared."""
    rows, cols, ops = synth.batch_operands(2, 4096, [("A", False), ("B", False), ("C", True)])
    shape = []
    zs, ss, _ = run_batch(fx, rows, cols, ops, True, repeat=2, tune="search", shape_out=shape)
    check(ops, rows, cols, zs, ss, range(len(rows)),
          report=f"schur_trans_accu/f32 batch of 4096 (shape {shape[0]})")
    assert np.all(np.isfinite(ss))


@pytest.mark.parametrize("shape", [(512, 2, 0, 0), (256, 8, 1, 0), (512, 4, 2, 0), (256, 2, 0, 0),
                                   (256, 4, 0, 1), (512, 2, 2, 1), (256, 8, 0, 1)])
def test_batch_launch_shapes(fx, shape):
    """Every batched launch shape the tuner picks from: 256/512 threads,
    2/3/4 stages, residency, 16- or 8-byte vectors per thread (pipeline 0 /
    1); direct and graph-captured."""
    rows, cols, ops = synth.batch_operands(7, 50, [("A", False), ("B", False), ("C", True)],
                                           lo=1, hi=260)
    for use_graph in (False, True):
        zs, ss, _ = run_batch(fx, rows, cols, ops, use_graph, repeat=2, shape=shape)
        check(ops, rows, cols, zs, ss, range(len(rows)))


def test_batch_autotune(fx, tmp_path, monkeypatch):
    monkeypatch.setenv("FX_TUNE_CACHE", str(tmp_path / "tune.json"))
    rows, cols, ops = synth.batch_operands(8, 64, [("A", False), ("B", False), ("C", True)],
                                           lo=16, hi=400)
    got = []
    zs, ss, _ = run_batch(fx, rows, cols, ops, True, tune="search", shape_out=got)
    check(ops, rows, cols, zs, ss, range(len(rows)))
    b, u, s, p = got[0]
    assert b in (256, 512) and u in (2, 4, 8) and s in (0, 1, 2) and p in (0, 1)
    again = []
    run_batch(fx, rows, cols, ops, True, tune="cache", shape_out=again)
    assert again[0] == got[0]


@pytest.mark.parametrize("storage", ["f64", "bf16"])
@pytest.mark.parametrize("shape", [(256, 2, 0, 0), (256, 4, 0, 1)])
def test_batch_other_storage_types(fx, storage, shape):
    """The batched kernel in FP64 (32-row tiles, 2-element chunks) and BF16
    (8-element chunks) storage, at both vector widths (pipeline 0: 16 bytes
    per thread per step, 1: 8 bytes); every matrix against the oracle at the
    storage type's tolerance."""
    import torch

    from harness import STORAGE_CODE, from_device, oracle_outputs, to_device, tolerance
    from oracle.compare import ErrorReport
    rows, cols, ops = synth.batch_operands(9, 24, [("A", False), ("B", False), ("C", True)],
                                           lo=1, hi=150, storage=storage)
    n = len(rows)
    tdt = torch.float64 if storage == "f64" else torch.bfloat16
    rdt = torch.float64 if storage == "f64" else torch.float32
    dev = {k: [to_device(ops[k][i]) for i in range(n)] for k in "ABC"}
    zs = [torch.full((max(int(r) * int(c), 1),), float("nan"), dtype=tdt, device="cuda")
          for r, c in zip(rows, cols)]
    S = torch.full((n,), float("nan"), dtype=rdt, device="cuda")
    items = (fx.BatchItem * n)()
    for i in range(n):
        it = items[i]
        for k, name in enumerate("ABC"):
            it.ptr[k] = dev[name][i].data_ptr()
        it.ptr[3] = zs[i].data_ptr()
        it.ptr[4] = S.data_ptr() + i * S.element_size()
        it.rows, it.cols = int(rows[i]), int(cols[i])
    h = fx.fx_expr_create("schur_trans_accu", STORAGE_CODE[storage])
    try:
        fx.fx_expr_set_launch_shape(h, *shape)
        for use_graph in (False, True):
            fx.fx_eval_batch(h, items, 0, use_graph)
            torch.cuda.synchronize()
            s_got = S.cpu().numpy().astype(np.float64)
            for i in range(n):
                r, c = int(rows[i]), int(cols[i])
                env = {k: ops[k][i] for k in "ABC"}
                ref = oracle_outputs("schur_trans_accu", env)
                z = from_device(zs[i][: r * c], storage).reshape(c, r).T if r * c else np.zeros((r, c))
                zr, zm = ref["Z"]
                tz = tolerance("schur_trans_accu", storage, "Z")
                rz = ErrorReport(storage, tz, "m").add(z, zr, mag=zm)
                assert rz.nonfinite == 0 and rz.err <= tz, (storage, shape, i, r, c, rz.err)
                v, sv = ref["s"]
                ts = tolerance("schur_trans_accu", storage, "s")
                rs = ErrorReport("f64" if storage == "f64" else "f32", ts, "m").add(
                    [s_got[i]], [v], mag=[sv])
                assert rs.nonfinite == 0 and rs.err <= ts, (storage, shape, i, "s", rs.err)
    finally:
        fx.fx_expr_destroy(h)
