"""Benchmark of fused expression evaluation on one GB300 (or N replicas).

Default workload (the JSON line printed with no flags): one step evaluates, on
four 8192 x 8192 column-major FP32 matrices X, Y, W, V drawn i.i.d. N(0, 1)
(seed 1),
    Z      = X % Y + sqrt(abs(W)) / (1 + exp(-V))
    colsum = sum(X % Y, 0)
    rowmax = max(abs(X - Y), 1)
    nrm    = norm(X - Y, 2)
each as one fused kernel. The metric is effective HBM bandwidth:
algorithmic bytes (every input element read once, every output written
once) per second. The inputs (256 MiB each) are larger than L2, so there is
no flush between iterations.

--workload selects the other measured configurations (same JSON fields):
  expr8192_f64   the default trees with FP64 storage
  small1024      Z = A%B + 3.5*exp(C) - trans(D) and s = accu(square(A-B)),
                 FP32 1024^2 (L2 flushed before every kernel, device-timed)
  prec16384_bf16 / prec16384_f16   the 1024^2 trees at 16384^2
  batch4096      Z = A%B + 0.5*trans(C), s = accu(Z) over 4096 matrices,
                 rows/cols log-uniform in [16, 2048], one graph-replayed launch
  loss8192_f32 / loss8192_bf16     L = accu(square(sigmoid(X%W + b) - Y))
                 forward and fused backward (dX, dW, db)
  suite10k       the Sec. 4 expressions at 10000^2 FP32: add-N, N = 2..16,
                 expr1, expr2, relu, sigmoid, swish, gelu

  prec16384_f16_clamped   prec16384_f16's Z with C's values capped at 9 (every
                 FP16 output finite)
  gemm8192_bf16 / gemm8192_f16   Z = sigmoid(X*Y/sqrt(K) + W) and Z = 2*X*Y^T at
                 M = N = K = 8192 on the tensor-core kernel (TFLOP/s), beside
                 the library GEMM plus the fused pass

With no flags, the line also carries "errors" (every output of the step
against the FP64 oracle, after the timed region) and "configs": each of
small1024, expr8192_f64, prec16384_bf16, prec16384_f16,
prec16384_f16_clamped, batch4096, loss8192_f32, loss8192_bf16, gemm8192_bf16
and gemm8192_f16 measured
the same way (autotuned, --config-steps timed steps), with its GB/s,
roofline fraction, speedup over the unfused baseline and errors.

--gpus N: N independent replicas (one process per GPU, torch.distributed.run);
value = bytes of all ranks / max elapsed time over ranks.
--impl reference: the FP64 CPU oracle, timed on a bounded sample of the
workload per step.
"""
from __future__ import annotations

import argparse
import csv
import datetime as dt
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused-expr effective HBM GB/s (% of GB300 peak) and speedup vs unfused per-op"

# DRAM traffic per launch of a dominant kernel from an ncu capture (bytes),
# valid only while the kernel sources hash to the recorded value.
TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on the first
    # timed launch of Z at 8192^2 FP32 (the flat kernel's summary under profiles/),
    # read + write per (threads per block, vectors per leaf) of the register
    # kernel k_flat, every shape the autotuner searches (pipelines 0 and 2 of
    # this four-leaf tree; the blocks-per-SM cap only changes the grid of the
    # same streaming loop). Reads are the 1,073,741,824 algorithmic bytes
    # within 0.02%; writes fall short of 268,435,456 by the part of Z still in
    # L2 when the launch ends.
    ("expr8192", "Z"): {"hash": "26d9b77dd5020077",
                        "bytes": {
                                  (128, 2): 1073773824 + 241745664,
                                  (128, 4): 1073779712 + 240940544,
                                  (128, 8): 1073778944 + 241056512,
                                  (256, 2): 1073772288 + 241765120,
                                  (256, 4): 1073889536 + 240781568,
                                  (256, 8): 1073779456 + 241166848,
                                  (512, 2): 1073836800 + 241808896,
                                  (512, 4): 1073789184 + 240969472,
                                  (512, 8): 1073901568 + 241073152}},
}

# FP64-pipe instructions per output element of FP64 trees (per lane: DFMA,
# DADD and DMUL each take one slot), counted with ncu
# (smsp__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on.sum over
# 4096^2 elements): exp, sqrt and division of the Z tree run as FMA
# sequences on the FP64 pipe, which on GB300 is slower than HBM.
FP64_PIPE_OPS = {("expr8192_f64", "Z"): 35}


def recorded_traffic(workload, dom, shape, source_hash):
    """DRAM bytes per launch recorded for the dominant tree, or None when the
    kernel sources changed since the capture, the launch shape (block,
    unroll, blocks/SM, pipeline) was not captured, or pipeline 1 selected the
    bulk-copy kernel instead of the register kernel."""
    tr = TRAFFIC.get((workload, dom))
    if not tr or tr["hash"] != source_hash:
        return None
    block, unroll, _, pipe = shape
    if pipe == 1:
        return None
    return tr["bytes"].get((block, unroll))


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("core.cuh", "expr.cuh", "plan.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2604_22242_gb300", "csrc", "fx", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_tensor_peak():
    """Dense BF16 tensor throughput (TFLOP/s) measured on this machine (burst: a
    kernel timed alone), else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons; keeps the samples
    whose timestamps fall inside [t0, t1] (host wall clock)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.p = index, None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self, t0, t1):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for r in csv.reader(io.StringIO(out)):
            if len(r) < 10:
                continue
            try:
                ts = dt.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(r[2]), float(r[3]), float(r[4]),
                             [r[6 + k].strip().lower() == "active" for k in range(4)]))
            except ValueError:
                continue
        inside = [x for x in rows if t0 - 0.05 <= x[0] <= t1 + 0.05] or rows
        reasons = sorted({names[k] for x in inside for k in range(4) if x[4][k]})
        return {"sm_mhz": statistics.median(x[1] for x in inside) if inside else None,
                "sm_max_mhz": max((x[2] for x in inside), default=None),
                "power_w_max": max((x[3] for x in inside), default=None),
                "reasons": reasons, "samples": len(inside)}


# ---------------------------------------------------------------- workloads

class Op:
    """One fused evaluation: a launch, its unfused twin, its algorithmic bytes,
    its elements (output elements, or the elements a reduction reduces) and
    (trees with a matrix product) its algorithmic flops."""

    def __init__(self, key, nbytes, launch, unfused=None, launches=None, flops=0, elems=0):
        self.key, self.bytes, self.launch, self.unfused, self.launches = (
            key, nbytes, launch, unfused, launches)
        self.flops = flops
        self.elems = elems


def _bind(fx, h, k, t, rows, cols, ld):
    fx.fx_expr_bind(h, k, t.data_ptr(), rows, cols, ld)


def _expr_ops(fx, torch, dev, sp, trees, storage, env, R, C, keep, check=True):
    """Ops for single-matrix trees. trees: [(name, key, input names, out kind)];
    out kind "Zs" is a matrix Z plus a scalar s from one launch. With check,
    the outputs are compared with the oracle after the timed region."""
    import numpy as np
    code = {"f32": fx.FX_F32, "f64": fx.FX_F64, "bf16": fx.FX_BF16, "f16": fx.FX_F16}[storage]
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16,
           "f16": torch.float16}[storage]
    rdt = torch.float64 if storage == "f64" else torch.float32
    es = {"f32": 4, "f64": 8, "bf16": 2, "f16": 2}[storage]
    rs = 8 if storage == "f64" else 4
    d = keep.get("inputs")
    if d is None:
        d = {}
        for k, b in env.items():
            if storage == "bf16":
                t = torch.from_numpy(b.data.view(np.int16)).view(torch.bfloat16)
            else:
                t = torch.from_numpy(b.data)
            d[k] = t.to(dev)
        keep["inputs"] = d
    ops = []
    for name, key, ins, kind in trees:
        h = fx.fx_expr_create(name, code)
        nb = 0
        for k, s in enumerate(ins):
            b = env[s]
            _bind(fx, h, k, d[s], b.rows, b.cols, b.ld)
            if s not in ins[:k]:          # a leaf read twice is read once (fusion)
                nb += b.rows * b.cols * {"f32": 4, "f64": 8, "bf16": 2, "f16": 2}[b.storage]
        if kind == "Z":
            o = torch.empty(R * C, dtype=tdt, device=dev)
            _bind(fx, h, len(ins), o, R, C, R)
            nb += R * C * es
        elif kind == "s":
            o = torch.empty(1, dtype=rdt, device=dev)
            _bind(fx, h, len(ins), o, 1, 1, 1)
            nb += rs
        elif kind == "Zs":
            o = (torch.empty(R * C, dtype=tdt, device=dev), torch.empty(1, dtype=rdt, device=dev))
            _bind(fx, h, len(ins), o[0], R, C, R)
            _bind(fx, h, len(ins) + 1, o[1], 1, 1, 1)
            nb += R * C * es + rs
        elif kind == "col":
            o = torch.empty(C, dtype=rdt, device=dev)
            _bind(fx, h, len(ins), o, 1, C, 1)
            nb += C * rs
        elif kind == "row":
            o = torch.empty(R, dtype=rdt, device=dev)
            _bind(fx, h, len(ins), o, R, 1, R)
            nb += R * rs
        keep[key] = (h, o)
        keep.setdefault("_handles", []).append(h)
        if check:
            keep.setdefault("trees", []).append((name, key, list(ins), kind))
        ops.append(Op(key, nb, (lambda h=h: fx.fx_eval(h, sp)),
                      (lambda h=h: fx.fx_eval_unfused(h, sp)),
                      (lambda h=h: fx.fx_expr_last_launches(h)), elems=R * C))
    return ops


def workload(name, fx, torch, dev, sp, keep, size=8192, count=4096):
    """(ops, config dict, dominant op key, flush_l2, dtype) for a workload."""
    import numpy as np
    import synth
    if name in ("expr8192", "expr8192_f64"):
        storage = "f64" if name.endswith("f64") else "f32"
        R = C = size
        env = synth.operands(1, [("X", R, C), ("Y", R, C), ("W", R, C), ("V", R, C)], storage,
                             "normal")
        trees = [("schur_sqrt_sigmoid", "Z", "XYWV", "Z"), ("schur_colsum", "colsum", "XY", "col"),
                 ("absdiff_rowmax", "rowmax", "XY", "row"), ("diff_norm", "nrm", "XY", "s")]
        cfg = {"workload": "X%Y+sqrt(abs(W))/(1+exp(-V)), sum(X%Y,0), max(abs(X-Y),1), "
                           f"norm(X-Y,2) at {R}x{C}", "rows": R, "cols": C,
               "inputs": "X,Y,W,V i.i.d. N(0,1), seed 1, column-major",
               "l2": "inputs larger than L2 (256 MiB each in FP32), no flush"}
        keep["env"] = env
        return _expr_ops(fx, torch, dev, sp, trees, storage, env, R, C, keep), cfg, "Z", False, storage
    if name in ("small1024", "prec16384_bf16", "prec16384_f16", "prec16384_f16_clamped"):
        storage = "f32" if name == "small1024" else name.split("_")[1]
        R = C = (1024 if name == "small1024" else 16384) if size == 8192 else size
        dist = "uniform" if name == "small1024" else "lognormal_signed"
        env = synth.operands(0, [("A", R, C), ("B", R, C), ("C", R, C), ("D", C, R)], storage, dist)
        inputs = f"A,B,C,D {dist}, seed 0, column-major"
        # Z and s in one pass over A, B, C, D; the two separate trees are
        # timed beside it ("separate_trees") for comparison
        trees = [("schur_exp_trans_sqdiff", "Zs", "ABCD", "Zs")]
        sep = [("schur_exp_trans", "Z_alone", "ABCD", "Z"), ("sqdiff_accu", "s_alone", "AB", "s")]
        if name.endswith("_clamped"):
            # C's values capped at 9: 3.5 exp(9) = 28361 stays finite in FP16
            c = env["C"]
            cap = synth.round_to_storage(np.array([9.0]), storage)[0]
            env["C"] = synth.Buffer(np.where(synth.to_f64(c.data, storage) > 9.0, cap, c.data),
                                    c.rows, c.cols, c.ld, storage)
            inputs += "; C capped at 9"
        cfg = {"workload": f"A%B+3.5*exp(C)-trans(D) and accu(square(A-B)) in one pass at {R}x{C}",
               "rows": R, "cols": C, "inputs": inputs,
               "l2": "L2 flushed before every kernel (256 MiB write), device-timed per kernel"
               if name == "small1024" else "inputs larger than L2, no flush"}
        keep["env"] = env
        ops = _expr_ops(fx, torch, dev, sp, trees, storage, env, R, C, keep)
        keep["alt_ops"] = _expr_ops(fx, torch, dev, sp, sep, storage, env, R, C, keep, check=False)
        return ops, cfg, "Zs", name == "small1024", storage
    if name == "batch4096":
        return batch_workload(fx, torch, dev, sp, keep, count)
    if name == "suite10k":
        R = C = 10000 if size == 8192 else size
        env = synth.operands(4, [(f"A{k}", R, C) for k in range(1, 17)], "f32", "uniform")
        env.update(synth.operands(5, [("P1", R, C), ("P2", R, C)], "f32", "positive"))
        env.update(synth.operands(6, [("Y64", R, C)], "f64", "normal"))
        trees = [(f"add{n}", f"add{n}", [f"A{k}" for k in range(1, n + 1)], "Z")
                 for n in range(2, 17)]
        trees += [("expr1", "expr1", ["A1", "A2"], "Z"),
                  ("expr2", "expr2", ["A1", "A2", "A3", "A4"], "Z"),
                  ("expr3", "expr3", ["P1", "Y64", "P2"], "Z"),
                  ("relu", "relu", ["A1"], "Z"), ("sigmoid", "sigmoid", ["A1"], "Z"),
                  ("swish", "swish", ["A1"], "Z"), ("gelu", "gelu", ["A1"], "Z")]
        cfg = {"workload": "Sec. 4 suite at 10000x10000 FP32: add-N (N=2..16), expr1, expr2, "
                           "expr3 (FP64 Y), relu, sigmoid, swish, gelu", "rows": R, "cols": C,
               "inputs": "A1..A16 U[-1,1], seed 4; P1, P2 U[0.5,2], seed 5; Y64 FP64 N(0,1), "
                         "seed 6; column-major",
               "l2": "inputs larger than L2 (400 MB each), no flush"}
        keep["env"] = env
        return _expr_ops(fx, torch, dev, sp, trees, "f32", env, R, C, keep), cfg, "add16", False, "f32"
    if name in ("loss8192_f32", "loss8192_bf16"):
        return loss_workload(fx, torch, dev, sp, keep, name.split("_")[1], size)
    if name in ("gemm8192_bf16", "gemm8192_f16"):
        return gemm_workload(fx, torch, dev, sp, keep, name.split("_")[1], size)
    raise SystemExit(f"unknown workload {name}")


def gemm_workload(fx, torch, dev, sp, keep, storage, size=8192):
    """Trees with one matrix product at M = N = K = size: Z = sigmoid(s X Y + W)
    (s = 1/sqrt(K), so the sigmoid is not saturated) and Fig. 1's Z = 2 X Y^T,
    on the tcgen05 kernel with the remainder in its epilogue (launch-shape
    pipeline 0); the same trees through the library GEMM and the fused pass
    (pipeline 2) are timed beside them."""
    import numpy as np
    import synth
    M = N = K = size
    env = synth.operands(7, [("X", M, K), ("Y", K, N), ("W", M, N), ("Yt", N, K)], storage,
                         "normal")
    code = fx.FX_BF16 if storage == "bf16" else fx.FX_F16
    tdt = torch.bfloat16 if storage == "bf16" else torch.float16
    d = {}
    for k, b in env.items():
        t = torch.from_numpy(b.data.view(np.int16)).view(tdt) if storage == "bf16" else \
            torch.from_numpy(b.data)
        d[k] = t.to(dev)
    keep["inputs"] = d
    keep["env"] = env
    flops = 2 * M * N * K
    trees = [("gemm_epilogue", "epilogue", ["X", "Y", "W"], [1.0 / K ** 0.5]),
             ("gemm_scale", "scale", ["X", "Yt"], [2.0])]

    def make(pipe, suffix, check):
        ops = []
        for name, key, ins, scal in trees:
            h = fx.fx_expr_create(name, code)
            for i, v in enumerate(scal):
                fx.fx_expr_set_scalar(h, i, v)
            nb = 0
            for k, sname in enumerate(ins):
                b = env[sname]
                fx.fx_expr_bind(h, k, d[sname].data_ptr(), b.rows, b.cols, b.ld)
                nb += b.rows * b.cols * 2
            z = torch.empty(M * N, dtype=tdt, device=dev)
            fx.fx_expr_bind(h, len(ins), z.data_ptr(), M, N, M)
            nb += M * N * 2
            fx.fx_expr_set_launch_shape(h, 256, 4, 0, pipe)
            keep[key + suffix] = (h, z)
            keep.setdefault("_handles", []).append(h)
            if check:
                keep.setdefault("gemm_checks", []).append((name, key, ins, scal))
            ops.append(Op(key + suffix, nb, (lambda h=h: fx.fx_eval(h, sp)),
                          (lambda h=h: fx.fx_eval_unfused(h, sp)),
                          (lambda h=h: fx.fx_expr_last_launches(h)), flops=flops,
                          elems=M * N))
        return ops

    ops = make(0, "", True)
    keep["alt_ops"] = make(2, "_library", False)
    keep["alt_what"] = ("the same trees through the library GEMM (cuBLAS) and the fused "
                        "element-wise pass (launch-shape pipeline 2)")
    keep["no_tune"] = True
    cfg = {"workload": f"Z=sigmoid(X*Y/sqrt(K)+W) and Z=2*X*Y^T at M=N=K={size} {storage}",
           "rows": M, "cols": N, "inner": K,
           "inputs": "X, Y, W, Y^T-operand N(0,1), seed 7, column-major",
           "l2": "operands 128 MiB each; a GEMM re-reads them from L2 by design, no flush"}
    return ops, cfg, "epilogue", False, storage


def batch_workload(fx, torch, dev, sp, keep, count=4096):
    import numpy as np
    import synth
    rows, cols, ops_ = synth.batch_operands(2, count, [("A", False), ("B", False), ("C", True)])
    n = len(rows)

    def arena(mats):
        offs, pos = [], 0
        for m in mats:
            offs.append(pos)
            pos += (m.data.size + 3) // 4 * 4
        host = np.zeros(pos, dtype=np.float32)
        for m, o in zip(mats, offs):
            host[o:o + m.data.size] = m.data
        return torch.from_numpy(host).to(dev), offs

    A, oa = arena(ops_["A"])
    B, ob = arena(ops_["B"])
    Cm, oc = arena(ops_["C"])
    # 64 matrices (seeded) plus the largest and the smallest are kept for the
    # oracle check after the timed region
    rng = np.random.default_rng(2)
    pick = sorted(set(rng.choice(n, 64, replace=False).tolist()) |
                  {int(np.argmax(rows * cols)), int(np.argmin(rows * cols))})
    keep["batch_sample"] = (pick, {k: [ops_[k][i] for i in pick] for k in "ABC"})
    del ops_
    oz, pos = [], 0
    for r, c in zip(rows, cols):
        oz.append(pos)
        pos += (int(r * c) + 3) // 4 * 4
    Z = torch.empty(pos, dtype=torch.float32, device=dev)
    S = torch.empty(n, dtype=torch.float32, device=dev)
    items = (fx.BatchItem * n)()
    for i in range(n):
        it = items[i]
        it.ptr[0] = A.data_ptr() + 4 * oa[i]
        it.ptr[1] = B.data_ptr() + 4 * ob[i]
        it.ptr[2] = Cm.data_ptr() + 4 * oc[i]
        it.ptr[3] = Z.data_ptr() + 4 * oz[i]
        it.ptr[4] = S.data_ptr() + 4 * i
        it.rows, it.cols = int(rows[i]), int(cols[i])
    h = fx.fx_expr_create("schur_trans_accu", fx.FX_F32)
    keep["batch"] = (A, B, Cm, Z, S, items, h)
    keep["batch_offsets"] = (oz, rows, cols)
    keep.setdefault("_handles", []).append(h)
    nel = int(np.sum(rows * cols))
    nbytes = 16 * nel + 4 * n
    # unfused and unbatched baseline: the same tree one operator per launch, matrix by matrix
    per = []
    for i in range(n):
        e = fx.fx_expr_create("schur_trans_accu", fx.FX_F32)
        r, c = int(rows[i]), int(cols[i])
        fx.fx_expr_bind(e, 0, items[i].ptr[0], r, c, r)
        fx.fx_expr_bind(e, 1, items[i].ptr[1], r, c, r)
        fx.fx_expr_bind(e, 2, items[i].ptr[2], c, r, c)
        fx.fx_expr_bind(e, 3, items[i].ptr[3], r, c, r)
        fx.fx_expr_bind(e, 4, items[i].ptr[4], 1, 1, 1)
        per.append(e)
    keep["per"] = per
    keep["_handles"].extend(per)

    def unfused():
        for e in per:
            fx.fx_eval_unfused(e, sp)

    op = Op("batch", nbytes, lambda: fx.fx_eval_batch(h, items, sp, True), unfused,
            lambda: fx.fx_expr_last_launches(h), elems=nel)
    cfg = {"workload": f"Z=A%B+0.5*trans(C), s=accu(Z) over {n} matrices, rows/cols "
                       "log-uniform [16,2048] seed 2", "matrices": n, "elements": nel,
           "l2": "working set 11.5 GB, no flush", "graph": True}
    return [op], cfg, "batch", False, "f32"


def loss_workload(fx, torch, dev, sp, keep, storage, size=8192):
    import numpy as np
    import synth
    R = C = size
    env = synth.operands(3, [("X", R, C), ("W", R, C), ("Y", R, C), ("b", R, 1)], storage,
                         "normal_half")
    tdt = torch.float32 if storage == "f32" else torch.bfloat16
    es = 4 if storage == "f32" else 2
    d = {}
    for k, b in env.items():
        t = torch.from_numpy(b.data.view(np.int16)).view(torch.bfloat16) if storage == "bf16" \
            else torch.from_numpy(b.data)
        d[k] = t.to(dev)
    code = fx.FX_F32 if storage == "f32" else fx.FX_BF16
    h = fx.fx_expr_create("sigmoid_sqloss", code)
    for k, s in enumerate("XWYb"):
        b = env[s]
        fx.fx_expr_bind(h, k, d[s].data_ptr(), b.rows, b.cols, b.ld)
    L = torch.empty(1, dtype=torch.float32, device=dev)
    fx.fx_expr_bind(h, 4, L.data_ptr(), 1, 1, 1)
    g = {s: torch.empty(R * C, dtype=tdt, device=dev) for s in "XW"}
    g["b"] = torch.empty(R, dtype=tdt, device=dev)
    ptrs = [g["X"].data_ptr(), g["W"].data_ptr(), 0, g["b"].data_ptr()]
    keep["loss"] = (d, L, g, h)
    keep["env"] = env
    keep.setdefault("_handles", []).append(h)
    fwd_bytes = 3 * R * C * es + R * es + 4
    bwd_bytes = 3 * R * C * es + R * es + 2 * R * C * es + R * es
    ops = [Op("forward", fwd_bytes, lambda: fx.fx_eval(h, sp), lambda: fx.fx_eval_unfused(h, sp),
              lambda: fx.fx_expr_last_launches(h), elems=R * C),
           Op("backward", bwd_bytes, lambda: fx.fx_eval_backward(h, 0, ptrs, sp), None,
              lambda: fx.fx_expr_last_launches(h), elems=R * C)]
    cfg = {"workload": f"L=accu(square(sigmoid(X%W+b.each_col)-Y)) forward and backward (dX,dW,db), "
                       f"{R}x{C} {storage}", "rows": R, "cols": C,
           "inputs": "X,W,Y,b N(0, sd 0.5), seed 3", "l2": "inputs larger than L2, no flush"}
    return ops, cfg, "backward", False, storage


# ---------------------------------------------------------------- ranks

def aggregate(ms_local, step_bytes, steps, world, dist=None, device="cpu"):
    """Whole-job timing over replicas: the slowest rank's timed region
    (max over ranks) and the bytes of all ranks over that time (GB/s)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * step_bytes * steps / (ms / 1e3) / 1e9


# ---------------------------------------------------------------- CPU oracle

ORACLE_TREES = {
    "Z": "(+ (% X Y) (/ (sqrt (abs W)) (+ 1.0 (exp (neg V)))))",
    "colsum": "(sum (% X Y) 0)",
    "rowmax": "(max (abs (- X Y)) 1)",
    "nrm": "(norm (- X Y))",
}


def cpu_oracle_time(R, cols, storage):
    """The oracle on an R x cols panel of the default workload: (s, bytes)."""
    import oracle
    import synth
    env = synth.operands(1, [("X", R, cols), ("Y", R, cols), ("W", R, cols), ("V", R, cols)],
                         storage, "normal")
    es = 8 if storage == "f64" else 4
    N = R * cols
    nbytes = 5 * N * es + (2 * N * es + cols * es) + (2 * N * es + R * es) + (2 * N * es + es)
    t0 = time.perf_counter()
    for tree in ORACLE_TREES.values():
        oracle.evaluate(tree, env)
    return time.perf_counter() - t0, nbytes


def _oracle_worker(a):
    R, cols, storage = a
    return cpu_oracle_time(R, cols, storage)


def cpu_oracle_time_all_cores(R, cols, storage, nproc):
    """The same oracle on nproc panels at once, one process per core
    (spawned, so no CUDA state is inherited): (wall s of the slowest, bytes)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc) as pool:
        pool.map(_oracle_worker, [(R, 8, storage)] * nproc)      # imports and warm-up
        res = pool.map(_oracle_worker, [(R, cols, storage)] * nproc)
    return max(t for t, _ in res), sum(b for _, b in res)


def run_reference(args, rank, world):
    if rank != 0:
        return
    R = 8192
    # the sample per step is sized so that warm-up and timed steps together
    # take about 100 s of CPU time (at most --ref-cols columns per step)
    t64, _ = cpu_oracle_time(R, 64, "f32")
    per_col = max(t64 / 64, 1e-6)
    budget = 100.0 / max(1, args.steps + args.warmup)
    cols = int(max(8, min(args.ref_cols, budget / per_col)))
    for _ in range(args.warmup):
        cpu_oracle_time(R, cols, "f32")
    tt, tb = 0.0, 0
    for _ in range(args.steps):
        t, b = cpu_oracle_time(R, cols, "f32")
        tt += t
        tb += b
    v = tb / tt / 1e9
    sample = (f"{R}x{cols} column panel of X,Y,W,V per step, all four trees, FP64 numpy "
              "tree walker, one thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * tt / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "X%Y+sqrt(abs(W))/(1+exp(-V)), sum(X%Y,0), max(abs(X-Y),1), "
                               "norm(X-Y,2) at 8192x8192", "sample_cols": cols,
                   "l2": "CPU run, no GPU"},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0}), flush=True)


# ---------------------------------------------------------------- oracle check leg
#
# After the timed region, each output of a step is compared with the FP64
# oracle (the checker: nothing here is timed, and no result of the library
# is computed by it). Element-wise outputs are compared at 2^16 seeded
# positions, reductions in full, the batch on 66 whole matrices, the
# gradients on 16 whole rows. Each entry carries the maximum scaled error
# under the oracle's running error bound sigma and under its magnitude
# scale m, the maximum plain relative error, the tolerance and the scale it
# gates on, and the counts of wrong non-finite outputs and of outputs that
# are expected to overflow the storage type.

# oracle trees of the compiled trees, over the workloads' input names
ORACLE_OF = {
    "schur_sqrt_sigmoid": "(+ (% X Y) (/ (sqrt (abs W)) (+ 1.0 (exp (neg V)))))",
    "schur_colsum": "(sum (% X Y) 0)",
    "absdiff_rowmax": "(max (abs (- X Y)) 1)",
    "diff_norm": "(norm (- X Y))",
    "schur_exp_trans": "(- (+ (% A B) (* 3.5 (exp C))) (t D))",
    "sqdiff_accu": "(accu (square (- A B)))",
    "schur_exp_trans_sqdiff": ("(- (+ (% A B) (* 3.5 (exp C))) (t D))", "(accu (square (- A B)))"),
    "schur_trans_accu": "(+ (% A B) (* 0.5 (t C)))",
    "sigmoid_sqloss": "(accu (square (- (sigmoid (+ (% X W) (each_col b))) Y)))",
    # the Sec. 4 suite, with the scalars the library's definitions default to
    "expr1": "(+ (* 2.0 (+ (t X) Y)) (* 2.0 (+ X (t Y))))",
    "expr2": "(+ (+ (* 0.75 A) (t (+ B C))) (log (pow D 2.0)))",
    "expr3": "(/ 1 (+ (% X (f32 Y)) (log (% (log (+ X 2)) W))))",
    "relu": "(% X (gt X 0.0))",
    "sigmoid": "(/ 1.0 (+ 1.0 (exp (neg X))))",
    "swish": "(/ X (+ 1 (exp (neg (* 1.0 X)))))",
    "gelu": "(% (/ X 2) (+ 1 (tanh (* 0.7978845608028654 (+ X (* 0.044715 (pow X 3)))))))",
}
# slot names of the oracle trees, in slot order, where they differ from the
# names of the workload's operands bound to them
ORACLE_SLOTS = {"expr1": ["X", "Y"], "expr2": ["A", "B", "C", "D"], "expr3": ["X", "Y", "W"],
                "relu": ["X"], "sigmoid": ["X"], "swish": ["X"], "gelu": ["X"]}
for _n in range(2, 17):
    _t = "A1"
    for _k in range(2, _n + 1):
        _t = f"(+ {_t} A{_k})"
    ORACLE_OF[f"add{_n}"] = _t


def _host64(t):
    import torch
    return t.detach().to(torch.float64).cpu().numpy()


def oracle_errors(keep, storage, n_sample=1 << 16):
    """{output key: error summary} for the outputs kept by a workload."""
    import concurrent.futures as cf

    import numpy as np
    import torch

    import oracle
    import synth
    from oracle import grad as ograd
    from oracle.compare import TOL_TRANS, ErrorReport, gate_scale, tolerance

    rst = "f64" if storage == "f64" else "f32"      # reductions come out in FP32 / FP64
    jobs = {}
    env = keep.get("env")
    for name, key, ins, kind in keep.get("trees", []):
        tree = ORACLE_OF[name]
        _, o = keep[key]
        tenv = env
        if name in ORACLE_SLOTS:
            tenv = {slot: env[i] for slot, i in zip(ORACLE_SLOTS[name], ins)}
        if kind == "Zs":     # Z of the first tree, s = accu of the second
            tree, side = tree
            o, osum = o
            g = _host64(osum).ravel()

            def sjob(side=side, g=g, tenv=tenv):
                v, sg = oracle.evaluate_sigma(side, tenv)
                m = oracle.evaluate_mag(side, tenv)
                return ErrorReport(rst, tolerance(side, storage), gate_scale(side)).add(
                    g, v.ravel(), sg.ravel(), m.ravel())
            jobs["s"] = sjob
            key, kind = "Z", "Z"
        if kind == "Z":
            first = env[ins[0]]
            R, C = first.rows, first.cols
            rng = np.random.default_rng(99)
            rr = rng.integers(0, R, n_sample)
            cc = rng.integers(0, C, n_sample)
            g = _host64(o[torch.from_numpy(rr + cc * R).to(o.device)])

            def zjob(tree=tree, rr=rr, cc=cc, g=g, tenv=tenv):
                v, sg = oracle.at_sigma(tree, tenv, rr, cc)
                m = oracle.at_mag(tree, tenv, rr, cc)
                return ErrorReport(storage, tolerance(tree, storage), gate_scale(tree)).add(
                    g, v, sg, m)
            jobs[key] = zjob
        else:
            g = _host64(o).ravel()

            def rjob(tree=tree, g=g, tenv=tenv):
                v, sg = oracle.evaluate_sigma(tree, tenv)
                m = oracle.evaluate_mag(tree, tenv)
                return ErrorReport(rst, tolerance(tree, storage), gate_scale(tree)).add(
                    g, v.ravel(), sg.ravel(), m.ravel())
            jobs[key] = rjob
    for name, key, ins, scal in keep.get("gemm_checks", []):
        _, z = keep[key]
        tree = {"gemm_epilogue": "(sigmoid (+ (* {s0} (* X Y)) W))",
                "gemm_scale": "(* {s0} (* X (t Y)))"}[name].format(s0=repr(float(scal[0])))
        X = env[ins[0]]
        M = X.rows
        N = env[ins[2]].cols if name == "gemm_epilogue" else env[ins[1]].rows
        rng = np.random.default_rng(17)
        rs = np.sort(rng.choice(M, 64, replace=False))
        cs = np.sort(rng.choice(N, 64, replace=False))
        g = _host64(z.view(N, M).T[torch.from_numpy(rs).to(z.device)][:, torch.from_numpy(cs).to(
            z.device)])

        def sub(b, rows_, cols_):
            full = b.data.reshape(b.cols, b.ld).T[: b.rows, :]
            part = np.ascontiguousarray(full[rows_][:, cols_].T).ravel()
            return synth.Buffer(part, len(rows_), len(cols_), len(rows_), b.storage)

        K_ = X.cols
        allk = np.arange(K_)
        if name == "gemm_epilogue":
            senv = {"X": sub(X, rs, allk), "Y": sub(env[ins[1]], allk, cs),
                    "W": sub(env[ins[2]], rs, cs)}
        else:
            senv = {"X": sub(X, rs, allk), "Y": sub(env[ins[1]], cs, allk)}

        def gjob(tree=tree, senv=senv, g=g):
            v, sg = oracle.evaluate_sigma(tree, senv)
            m = oracle.evaluate_mag(tree, senv)
            return ErrorReport(storage, tolerance(tree, storage), gate_scale(tree)).add(g, v, sg, m)
        jobs[key] = gjob
    if "loss" in keep:
        tree = ORACLE_OF["sigmoid_sqloss"]
        _, L, grads, _ = keep["loss"]
        lv = _host64(L)

        def fjob():
            v, sg = oracle.evaluate_sigma(tree, env)
            m = oracle.evaluate_mag(tree, env)
            return ErrorReport("f32", tolerance(tree, storage), gate_scale(tree)).add(
                lv, v.ravel(), sg.ravel(), m.ravel())
        jobs["forward"] = fjob
        R = env["X"].rows
        rows = np.sort(np.random.default_rng(3).choice(R, 16, replace=False))
        ghost = {k: t for k, t in grads.items()}

        def bjob():
            ref = ograd.gradient_sigma(tree, env, 1.0, rows=rows)
            # gradients are element-wise outputs of the reverse pass, stored
            # in the storage type and held to its bound through sigmoid
            rep = ErrorReport(storage, TOL_TRANS[storage], "sigma")
            for s_, (idx, v, sg) in ref.items():
                if s_ in ghost:
                    g = _host64(ghost[s_][torch.from_numpy(idx).to(ghost[s_].device)])
                    rep.add(g, v, sg)
            return rep
        jobs["backward"] = bjob
    if "batch" in keep:
        tree = ORACLE_OF["schur_trans_accu"]
        pick, mats = keep["batch_sample"]
        _, _, _, Z, S, _, _ = keep["batch"]
        oz, rows, cols = keep["batch_offsets"]
        Sh = _host64(S)
        zs = {}
        for j, i in enumerate(pick):
            r, c = int(rows[i]), int(cols[i])
            zs[i] = _host64(Z[oz[i]:oz[i] + r * c]).reshape(c, r).T

        def bzjob():
            rep = ErrorReport("f32", tolerance(tree, "f32"), gate_scale(tree))
            for j, i in enumerate(pick):
                e = {k: mats[k][j] for k in "ABC"}
                v, sg = oracle.evaluate_sigma(tree, e)
                rep.add(zs[i], v, sg, oracle.evaluate_mag(tree, e))
            return rep

        def bsjob():
            t = f"(accu {tree})"
            rep = ErrorReport("f32", tolerance(t, "f32"), gate_scale(t))
            for j, i in enumerate(pick):
                e = {k: mats[k][j] for k in "ABC"}
                v, sg = oracle.evaluate_sigma(t, e)
                rep.add([Sh[i]], v.ravel(), sg.ravel(), oracle.evaluate_mag(t, e).ravel())
            return rep
        jobs["batch_Z"] = bzjob
        jobs["batch_s"] = bsjob
    out = {}
    with cf.ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        futs = {k: ex.submit(f) for k, f in jobs.items()}
        for k, f in futs.items():
            d = f.result().as_dict()
            d["ok"] = (d["nonfinite"] == 0 and
                       (d["max_scaled_err_m"] if d["gate"] == "m" else
                        d["max_scaled_err_sigma"]) <= d["tol"])
            out[k] = d
    return out


# ---------------------------------------------------------------- GPU run

def tune_workload(fx, args, keep, ops, cfg, sp):
    """Launch shapes: fixed by --shape, else every tree autotuned (fx_tune
    search; the unfused baseline keeps the library's default shapes), and the
    batch by fx_tune_batch. Returns the expression handles by op key."""
    keys = [o.key for o in ops]
    handles = {key: val[0] for key, val in keep.items()
               if isinstance(val, tuple) and len(val) == 2 and key in keys}
    if "loss" in keep:
        handles["loss"] = keep["loss"][3]
    if args.shape:
        cfg["launch_shape"] = args.shape
        for h in handles.values():
            fx.fx_expr_set_launch_shape(h, *[int(v) for v in args.shape.split(",")])
    elif not args.no_tune and handles:
        for h in handles.values():
            fx.fx_tune(h, "search", sp)
        cfg["launch_shape"] = {k: "autotuned: block %d, unroll %d, blocks/SM %d, pipeline %d"
                               % tuple(fx.fx_expr_launch_shape(h)) for k, h in handles.items()}
    if "batch" in keep:
        hb, items = keep["batch"][6], keep["batch"][5]
        fx.fx_tune_batch(hb, items, "search", sp)
        cfg["launch_shape"] = "autotuned: block %d, unroll %d, blocks/SM %d, pipeline %d" % tuple(
            fx.fx_expr_launch_shape(hb))
    return handles


def timed_steps(torch, stream, ops, K, W, fl, before=None, after=None):
    """W untimed steps, then exactly K timed steps on `stream`: per-op
    CUDA-event times (ms) of every launch, the whole region's device time
    (ms), the kernel launches counted and the host wall-clock bounds of the
    region. `before`/`after` run around the region (clocks, barriers)."""
    for _ in range(W):
        for o in ops:
            fl()
            o.launch()
    torch.cuda.synchronize()
    ev = {o.key: [] for o in ops}
    if before:
        before()
    torch.cuda.synchronize()
    t_start = time.time()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    launches = 0
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
    for _ in range(K):
        for o in ops:
            fl()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            o.launch()
            b.record(stream)
            ev[o.key].append((a, b))
            launches += o.launches() if o.launches else 1
    t1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t_end = time.time()
    if after:
        after()
    per_all = {k: [a.elapsed_time(b) for a, b in v] for k, v in ev.items()}
    return per_all, t0.elapsed_time(t1), launches, t_start, t_end


def unfused_steps(torch, stream, ops, K, fl):
    """Mean CUDA-event time (ms) of the unfused baseline of every op that has one."""
    uops = [o for o in ops if o.unfused]
    uk = max(3, min(K, 20))
    for o in uops:
        o.unfused()
    torch.cuda.synchronize()
    uev = {o.key: [] for o in uops}
    for _ in range(uk):
        for o in uops:
            fl()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            o.unfused()
            b.record(stream)
            uev[o.key].append((a, b))
    torch.cuda.synchronize()
    return {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in uev.items()}


def refresh_outputs(torch, ops):
    """The unfused baseline writes the same output buffers: run every fused
    op once more, so that the oracle check reads what the fused path wrote."""
    for o in ops:
        o.launch()
    torch.cuda.synchronize()


def release(fx, torch, keep):
    """Frees a workload's expression objects and device buffers."""
    torch.cuda.synchronize()
    for h in keep.get("_handles", []):
        fx.fx_expr_destroy(h)
    keep.clear()
    torch.cuda.empty_cache()


# the other measured configurations, reported in the default line's "configs"
EXTRA_CONFIGS = ["small1024", "expr8192_f64", "prec16384_bf16", "prec16384_f16",
                 "prec16384_f16_clamped", "batch4096", "loss8192_f32", "loss8192_bf16",
                 "gemm8192_bf16", "gemm8192_f16"]


def run_config(args, name, fx, torch, dev, stream, sp, peak, K, W):
    """One configuration measured as the default line is (autotuned, K timed
    steps after W warm-up steps, CUDA events), its unfused baseline, and its
    outputs' errors against the oracle (after the timed region)."""
    keep = {}
    ops, cfg, dom, flush, storage = workload(name, fx, torch, dev, sp, keep, 8192, args.count)
    try:
        if not keep.get("no_tune"):
            tune_workload(fx, args, keep, ops, cfg, sp)
        flush_buf = torch.empty(64 << 20, dtype=torch.float32, device=dev) if flush else None

        def fl():
            if flush_buf is not None:
                flush_buf.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            per_all, ms, launches, _, _ = timed_steps(torch, stream, ops, K, W, fl)
            u_ms = unfused_steps(torch, stream, ops, K, fl)
            alt = None
            if keep.get("alt_ops"):
                aops = keep["alt_ops"]
                for h in [keep[o.key][0] for o in aops]:
                    if not args.no_tune and not args.shape and not keep.get("no_tune"):
                        fx.fx_tune(h, "search", sp)
                a_all, a_ms, _, _, _ = timed_steps(torch, stream, aops, K, W, fl)
                if flush:
                    a_ms = K * sum(statistics.mean(v) for v in a_all.values())
                a_bytes = sum(o.bytes for o in aops)
                alt = {"what": keep.get("alt_what",
                                        "the same results from separate trees, one launch each"),
                       "ms_per_step": round(a_ms / K, 4), "bytes_per_step": a_bytes,
                       "launches_per_step": len(aops),
                       "gbs": round(a_bytes * K / (a_ms / 1e3) / 1e9, 2),
                       "per_op_ms": {k: round(statistics.mean(v), 4) for k, v in a_all.items()}}
                a_flops = sum(o.flops for o in aops)
                if a_flops:
                    alt["tflops"] = round(a_flops * K / (a_ms / 1e3) / 1e12, 1)
        per_ms = {k: statistics.mean(v) for k, v in per_all.items()}
        if flush:
            ms = K * sum(per_ms.values())
        step_bytes = sum(o.bytes for o in ops)
        dom_op = next(o for o in ops if o.key == dom)
        dom_gbs = dom_op.bytes / per_ms[dom] / 1e6
        fused_u = sum(per_ms[k] for k in u_ms)
        out = {
            "workload": cfg["workload"], "dtype": storage, "steps": K, "warmup": W,
            "value": round(step_bytes * K / (ms / 1e3) / 1e9, 2), "unit": "GB/s",
            "ms_per_step": round(ms / K, 4), "pct_of_peak": round(100 * step_bytes * K / (ms / 1e3) / 1e9 / peak, 2),
            "vs_unfused": round(sum(u_ms.values()) / fused_u, 3) if u_ms else None,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(dom_gbs, 2),
                         "peak": peak, "unit": "GB/s", "frac": round(dom_gbs / peak, 4),
                         "alg_bytes_per_launch": dom_op.bytes,
                         "avg_launch_ms": round(per_ms[dom], 4)},
            "per_op": {k: {"ms": round(per_ms[k], 4), "bytes": next(o.bytes for o in ops if o.key == k),
                           "gbs": round(next(o.bytes for o in ops if o.key == k) / per_ms[k] / 1e6, 1),
                           "gelems_per_s": round(next(o.elems for o in ops if o.key == k) / per_ms[k] / 1e6, 2),
                           "unfused_ms": round(u_ms[k], 4) if k in u_ms else None}
                       for k in per_ms},
            "gpu_launches": launches, "launch_shape": cfg.get("launch_shape"), "l2": cfg["l2"],
            "inputs": cfg.get("inputs"),
        }
        refresh_outputs(torch, ops)
        flops = sum(o.flops for o in ops)
        if flops:
            tpeak, tkind = measured_tensor_peak()
            t_dom = dom_op.flops / (per_ms[dom] / 1e3) / 1e12
            out["value"] = round(flops * K / (ms / 1e3) / 1e12, 1)
            out["unit"] = "TFLOP/s"
            out.pop("pct_of_peak", None)
            out["roofline"] = {"bound": "tensor", "kernel": dom, "achieved": round(t_dom, 1),
                               "peak": tpeak, "peak_kind": tkind + " (bf16 dense, burst)",
                               "unit": "TFLOP/s", "frac": round(t_dom / tpeak, 4),
                               "alg_flops_per_launch": dom_op.flops,
                               "avg_launch_ms": round(per_ms[dom], 4)}
            for k in out["per_op"]:
                o = next(o for o in ops if o.key == k)
                out["per_op"][k]["tflops"] = round(o.flops / (per_ms[k] / 1e3) / 1e12, 1)
        if alt:
            out["separate_trees" if not flops else "library_gemm"] = alt
        if (name, dom) in FP64_PIPE_OPS:
            alu = fp64_roofline(fx, sp, name, dom, dom_op, per_ms[dom], peak, storage, cfg)
            if alu:
                out["roofline_alu"] = alu
        out["errors"] = oracle_errors(keep, storage)
        return out
    finally:
        release(fx, torch, keep)


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    import paper_2604_22242_gb300 as fx

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sp = int(stream.cuda_stream)
    keep = {}
    ops, cfg, dom, flush, storage = workload(args.workload, fx, torch, dev, sp, keep, args.size,
                                            args.count)
    handles = {} if keep.get("no_tune") else tune_workload(fx, args, keep, ops, cfg, sp)
    flush_buf = torch.empty(64 << 20, dtype=torch.float32, device=dev) if flush else None
    torch.cuda.synchronize()
    step_bytes = sum(o.bytes for o in ops)
    K = args.steps

    def fl():
        if flush_buf is not None:
            flush_buf.zero_()

    clk = Clocks(local)

    def before():
        clk.start()
        time.sleep(0.4)
        if world > 1:
            dist.barrier()

    def after():
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        per_all, ms, launches, t_start, t_end = timed_steps(torch, stream, ops, K, args.warmup, fl,
                                                            before, after)
        clocks = clk.stop(t_start, t_end)
        per_ms = {k: statistics.mean(v) for k, v in per_all.items()}
        if flush:   # device time of the kernels alone (flushes excluded)
            ms = K * sum(per_ms.values())
        # unfused baseline: the same step, one kernel per operator
        u_ms = unfused_steps(torch, stream, ops, K, fl)
        e2e = None
        if args.workload in ("expr8192", "expr8192_f64"):
            e2e = e2e_run(fx, torch, stream, sp, keep, storage, K, args.size)

    fused_u = sum(per_ms[k] for k in u_ms)
    ms, value = aggregate(ms, step_bytes, K, world, dist, device=dev)
    if rank != 0:
        return
    peak, peak_kind = measured_peak()
    dom_op = next(o for o in ops if o.key == dom)
    z_gbs = dom_op.bytes / (per_ms[dom] / 1e3) / 1e9
    traffic = None
    if dom in handles:
        traffic = recorded_traffic(args.workload, dom, fx.fx_expr_launch_shape(handles[dom]),
                                   kernel_source_hash())
    cpu = cpu_all = None
    if world == 1 and args.workload == "expr8192" and args.size == 8192 and not args.no_cpu:
        t_cpu, b_cpu = cpu_oracle_time(8192, args.cpu_cols, "f32")
        cpu = {"value": round(b_cpu / t_cpu / 1e9, 4), "unit": "GB/s", "cores": 1,
               "kind": "oracle",
               "sample": f"8192x{args.cpu_cols} column panel of X,Y,W,V, all four trees, "
                         "FP64 numpy tree walker, one thread"}
        ncores = os.cpu_count() or 1
        if ncores > 1:
            t_par, b_par = cpu_oracle_time_all_cores(8192, max(1, args.cpu_cols // 4), "f32", ncores)
            cpu_all = {"value": round(b_par / t_par / 1e9, 4), "unit": "GB/s", "cores": ncores,
                       "kind": "oracle",
                       "sample": f"{ncores} processes, each an 8192x{max(1, args.cpu_cols // 4)} "
                                 "panel, all four trees; bytes of all panels over the slowest"}
    cfg["parallelism"] = f"replicas x{world}"
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(ms / K, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": storage,
        "data": "synthetic", "config": cfg,
        "pct_of_peak": round(100 * value / world / peak, 2),
        "pct_of_8tbs_spec": round(100 * value / world / 8000, 2),
        "vs_unfused": round(sum(u_ms.values()) / fused_u, 3) if u_ms else None,
        "per_op": {k: {"ms": round(per_ms[k], 4), "median_ms": round(statistics.median(per_all[k]), 4),
                       "min_ms": round(min(per_all[k]), 4),
                       "bytes": next(o.bytes for o in ops if o.key == k),
                       "gbs": round(next(o.bytes for o in ops if o.key == k) / per_ms[k] / 1e6, 1),
                       "gelems_per_s": round(next(o.elems for o in ops if o.key == k) / per_ms[k] / 1e6, 2),
                       "unfused_ms": round(u_ms[k], 4) if k in u_ms else None}
                   for k in per_ms},
        "roofline": {"bound": "hbm", "achieved": round(z_gbs, 2), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(z_gbs / peak, 4),
                     "traffic": traffic, "kernel": dom,
                     "alg_bytes_per_launch": dom_op.bytes, "avg_launch_ms": round(per_ms[dom], 4)},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if cpu_all:
        line["cpu_baseline_all_cores"] = cpu_all
    step_flops = sum(o.flops for o in ops)
    if step_flops:   # trees with a matrix product: TFLOP/s against the tensor peak
        tpeak, tkind = measured_tensor_peak()
        t_dom = dom_op.flops / (per_ms[dom] / 1e3) / 1e12
        line["metric"] = "fused matrix-product trees TFLOP/s (% of the measured BF16 tensor peak)"
        line["value"] = round(value * 1e9 / step_bytes * step_flops / 1e12, 1)
        line["unit"] = "TFLOP/s"
        line["pct_of_peak"] = round(100 * line["value"] / world / tpeak, 2)
        line.pop("pct_of_8tbs_spec", None)
        line["roofline"] = {"bound": "tensor", "kernel": dom, "achieved": round(t_dom, 1),
                            "peak": tpeak, "peak_kind": tkind + " (bf16 dense, burst)",
                            "unit": "TFLOP/s", "frac": round(t_dom / tpeak, 4), "traffic": None,
                            "alg_flops_per_launch": dom_op.flops,
                            "avg_launch_ms": round(per_ms[dom], 4)}
        for k in line["per_op"]:
            o = next(o for o in ops if o.key == k)
            line["per_op"][k]["tflops"] = round(o.flops / (per_ms[k] / 1e3) / 1e12, 1)
    if (args.workload, dom) in FP64_PIPE_OPS:
        alu = fp64_roofline(fx, sp, args.workload, dom, dom_op, per_ms[dom], peak, storage, cfg)
        if alu:
            line["roofline"] = alu
    if e2e:
        line["e2e"] = e2e
    if not args.no_check:
        with torch.cuda.stream(stream):
            refresh_outputs(torch, ops)
        line["errors"] = oracle_errors(keep, storage)
    if world == 1 and args.workload == "expr8192" and args.size == 8192 and not args.no_configs:
        release(fx, torch, keep)
        line["configs"] = {}
        for name in EXTRA_CONFIGS:
            line["configs"][name] = run_config(args, name, fx, torch, dev, stream, sp, peak,
                                               args.config_steps, 3)
    print(json.dumps(line), flush=True)


def fp64_roofline(fx, sp, workload, dom, dom_op, ms, hbm_peak, storage, cfg):
    """The ALU roofline of an FP64 tree when it binds before HBM: FP64-pipe
    instructions per second (ncu count per element x elements / kernel time)
    against the FMA rate measured now on this GPU (fx_fp64_fma_rate)."""
    es = 8 if storage == "f64" else 4
    n_el = cfg["rows"] * cfg["cols"]
    ops = FP64_PIPE_OPS[(workload, dom)] * n_el
    fma_rate = fx.fx_fp64_fma_rate(sp) / 2.0          # FMA (pipe slots) per second
    t_alu = ops / fma_rate
    t_hbm = dom_op.bytes / (hbm_peak * 1e9)
    if t_alu <= t_hbm:
        return None
    achieved = ops / (ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(fma_rate / 1e9, 2),
            "peak_kind": "measured (fx_fp64_fma_rate, FP64 FMA chains on every SM)",
            "unit": "G FP64-pipe op/s", "frac": round(achieved * 1e9 / fma_rate, 4),
            "traffic": None, "kernel": dom,
            "alg_ops_per_launch": ops, "ops_per_element": FP64_PIPE_OPS[(workload, dom)],
            "avg_launch_ms": round(ms, 4),
            "hbm_frac": round(dom_op.bytes / (ms / 1e3) / 1e9 / hbm_peak, 4)}


def e2e_run(fx, torch, stream, sp, keep, storage, K, size):
    """Same step through fx_eval_host: the four inputs copied in from pinned
    host memory and every output copied back, each step."""
    env = keep["env"]
    d = keep["inputs"]
    host = {k: torch.from_numpy(env[k].data).pin_memory() for k in "XYWV"}
    hz_t, hz = keep["Z"][1], None
    hz = torch.empty(hz_t.numel(), dtype=hz_t.dtype).pin_memory()
    small = {k: (keep[k][1], torch.empty(keep[k][1].numel(), dtype=keep[k][1].dtype).pin_memory())
             for k in ("colsum", "rowmax", "nrm")}
    hin = [host[s].data_ptr() for s in "XYWV"]

    def step():
        fx.fx_eval_host(keep["Z"][0], hin, [hz.data_ptr()], sp)
        for k, (dev_t, host_t) in small.items():
            fx.fx_eval(keep[k][0], sp)
            host_t.copy_(dev_t, non_blocking=True)

    step()
    torch.cuda.synchronize()
    ek = max(3, min(K, 20))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(ek):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ems = e0.elapsed_time(e1) / ek
    es = 8 if storage == "f64" else 4
    R = C = size
    N = R * C
    step_bytes = 5 * N * es + (2 * N * es + C * es) + (2 * N * es + R * es) + (2 * N * es + es)
    return {"value": round(step_bytes / (ems / 1e3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": 4 * N * es, "d2h_bytes_per_step": N * es + (R + C + 1) * es,
            "ms_per_step": round(ems, 3),
            "path": "fx_eval_host (pinned host inputs in, Z out) + 3 fx_eval + small D2H reads"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="expr8192",
                    choices=["expr8192", "expr8192_f64", "small1024", "prec16384_bf16",
                             "prec16384_f16", "prec16384_f16_clamped", "batch4096",
                             "loss8192_f32", "loss8192_bf16", "suite10k", "gemm8192_bf16",
                             "gemm8192_f16"])
    ap.add_argument("--size", type=int, default=8192,
                    help="rows = cols of the expr8192 and loss8192 workloads (other values than "
                         "8192 also resize prec16384_* and suite10k, for profiling)")
    ap.add_argument("--count", type=int, default=4096, help="matrices of the batch4096 workload")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default launch shapes (no autotuning)")
    ap.add_argument("--shape", default="",
                    help="fixed launch shape block,unroll,blocks_per_sm,pipeline for every tree")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the comparison of the outputs with the oracle")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: skip the other configurations' entries")
    ap.add_argument("--config-steps", type=int, default=10,
                    help="timed steps of each other configuration in the default line")
    ap.add_argument("--cpu-cols", type=int, default=4096)
    ap.add_argument("--ref-cols", type=int, default=512)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
