"""Test harness: runs a compiled tree through the C ABI on synth inputs and
compares it with the FP64 oracle using the scaled error metric of
``oracle.compare``:

err_i = |gpu_i - oracle_i| / max(scale_i, |oracle_i|, tiny)

where the scale is the oracle's magnitude scale m (oracle.at_mag) for trees
of sums, products and scalars, and its running error bound sigma
(oracle.at_sigma) for trees with transcendentals, divisions or matrix
products (oracle.compare.gate_scale). Outputs whose oracle value overflows
the storage type must come out as an infinity of the same sign and are left
out of the maximum; for FP16 outputs below the smallest normal the check is
absolute (2^-24).
"""
from __future__ import annotations

import numpy as np

import oracle
import synth
from oracle.compare import MAXFIN, TINY, ErrorReport, gate_scale, scaled_error  # noqa: F401
from oracle.compare import tolerance as tolerance_of

STORAGE_CODE = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3}

# Oracle trees for the compiled expressions (written from the paper's
# notation, independently of the library's own formula strings).
TREES = {
    "schur_exp_trans": "(- (+ (% A B) (* {s0} (exp C))) (t D))",
    "sqdiff_accu": "(accu (square (- A B)))",
    "schur_sqrt_sigmoid": "(+ (% X Y) (/ (sqrt (abs W)) (+ {s0} (exp (neg V)))))",
    "schur_colsum": "(sum (% X Y) 0)",
    "absdiff_rowmax": "(max (abs (- X Y)) 1)",
    "diff_norm": "(norm (- X Y))",
    "schur_trans_accu": "(+ (% A B) (* {s0} (t C)))",
    # two results over the same leaves: Z (this tree) and s (SIDE_SUM below)
    "schur_exp_trans_sqdiff": "(- (+ (% A B) (* {s0} (exp C))) (t D))",
    "sigmoid_sqloss": "(accu (square (- (sigmoid (+ (% X W) (each_col b))) Y)))",
    "expr1": "(+ (* {s0} (+ (t X) Y)) (* {s0} (+ X (t Y))))",
    "expr2": "(+ (+ (* {s0} A) (t (+ B C))) (log (pow D {s1})))",
    "relu": "(% X (gt X {s0}))",
    "sigmoid": "(/ {s0} (+ {s0} (exp (neg X))))",
    "swish": "(/ X (+ 1 (exp (neg (* {s0} X)))))",
    "gelu": "(% (/ X 2) (+ 1 (tanh (* {s0} (+ X (* {s1} (pow X 3)))))))",
    "sum_schur": "(% (+ A B) (+ C D))",
    "expr3": "(/ 1 (+ (% X (f32 Y)) (log (% (log (+ X 2)) W))))",
    # matrix products (Fig. 1, a product with an element-wise remainder, Sec. 4 chain)
    "gemm_scale": "(* {s0} (* X (t Y)))",
    "gemm_epilogue": "(sigmoid (+ (* {s0} (* X Y)) W))",
    "chain": "(* (* (* A B) C) D)",
}
for _n in range(2, 17):
    _t = "A1"
    for _k in range(2, _n + 1):
        _t = f"(+ {_t} A{_k})"
    TREES[f"add{_n}"] = _t
# the second tree of a two-result definition, summed into s
SIDE_SUM = {"schur_exp_trans_sqdiff": "(accu (square (- A B)))"}
DEFAULT_SCALARS = {"schur_exp_trans": [3.5], "schur_exp_trans_sqdiff": [3.5], "schur_sqrt_sigmoid": [1.0],
                   "schur_trans_accu": [0.5], "expr1": [2.0], "expr2": [0.75, 2.0], "relu": [0.0],
                   "sigmoid": [1.0], "swish": [1.0], "gelu": [0.7978845608028654, 0.044715],
                   "gemm_scale": [2.0], "gemm_epilogue": [0.5]}
SLOTS = {
    "schur_exp_trans": ["A", "B", "C", "D"],
    "schur_exp_trans_sqdiff": ["A", "B", "C", "D"],
    "sqdiff_accu": ["A", "B"],
    "schur_sqrt_sigmoid": ["X", "Y", "W", "V"],
    "schur_colsum": ["X", "Y"],
    "absdiff_rowmax": ["X", "Y"],
    "diff_norm": ["X", "Y"],
    "schur_trans_accu": ["A", "B", "C"],
    "sigmoid_sqloss": ["X", "W", "Y", "b"],
    "expr1": ["X", "Y"], "expr2": ["A", "B", "C", "D"], "relu": ["X"], "sigmoid": ["X"],
    "swish": ["X"], "gelu": ["X"], "sum_schur": ["A", "B", "C", "D"],
    "gemm_scale": ["X", "Y"], "gemm_epilogue": ["X", "Y", "W"], "chain": ["A", "B", "C", "D"],
    "expr3": ["X", "Y", "W"],
}
for _n in range(2, 17):
    SLOTS[f"add{_n}"] = [f"A{_k}" for _k in range(1, _n + 1)]
TRANSPOSED = {"schur_exp_trans": {"D"}, "schur_exp_trans_sqdiff": {"D"}, "schur_trans_accu": {"C"}, "expr2": {"B", "C"}}
VECTORS = {"sigmoid_sqloss": {"b"}}

def tree_of(name, scalars=None):
    s = scalars if scalars is not None else DEFAULT_SCALARS.get(name, [])
    return TREES[name].format(**{f"s{i}": repr(float(v)) for i, v in enumerate(s)})


def specs_for(name, R, C):
    out = []
    for s in SLOTS[name]:
        if s in TRANSPOSED.get(name, ()):
            out.append((s, C, R))
        elif s in VECTORS.get(name, ()):
            out.append((s, R, 1))
        else:
            out.append((s, R, C))
    return out


def tolerance(name, storage, output="Z"):
    """The bound of output `output` ("Z", or "s"/"v" for a reduced output)."""
    return tolerance_of(tree_of(name), storage, reduction=output != "Z")


# ---------------------------------------------------------------- device side

def to_device(buf: synth.Buffer, pad: int = 0):
    """Flat device copy of a synth buffer (plus `pad` trailing elements)."""
    import torch
    data = buf.data
    if buf.storage == "bf16":
        t = torch.from_numpy(data.view(np.int16).copy()).view(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(data))
    if pad:
        t = torch.cat([t, torch.zeros(pad, dtype=t.dtype)])
    return t.cuda()


def from_device(t, storage) -> np.ndarray:
    import torch
    if t.dtype == torch.bfloat16:
        return synth.to_f64(t.view(torch.int16).cpu().numpy().view(np.uint16), "bf16")
    return t.double().cpu().numpy()


def torch_dtype(storage):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16,
            "f16": torch.float16}[storage]


def canary_buffer(n, dtype, guard=64):
    import torch
    t = torch.empty(n + guard, dtype=dtype, device="cuda")
    t.fill_(float("nan"))
    return t


def check_canary(t, start, guard=64):
    import torch
    tail = t[start:start + guard]
    assert bool(torch.isnan(tail.float()).all()), "write past the end of an output"


def run(fx, name, storage, env, R, C, ldz=None, offset=0, unfused=False, scalars=None,
        stream=None, shape=None, tune=None):
    """Evaluates `name` on device copies of `env`; returns the outputs as FP64.

    shape: (block, unroll, blocks_per_sm, pipeline) to fix the launch shape;
    tune: "search" or "cache" to run the autotuner on the bound buffers first
    (the chosen shape is returned under "_shape")."""
    import torch
    h = fx.fx_expr_create(name, STORAGE_CODE[storage])
    try:
        n_in, n_out, n_scal, kind = fx.fx_expr_info(h)
        if shape is not None:
            fx.fx_expr_set_launch_shape(h, *shape)
            assert tuple(fx.fx_expr_launch_shape(h)) == tuple(shape)
        if scalars is not None:
            for i, v in enumerate(scalars):
                fx.fx_expr_set_scalar(h, i, v)
        keep = []
        for k, s in enumerate(SLOTS[name]):
            b = env[s]
            t = to_device(b, pad=offset)
            if offset:
                t = t.roll(offset)  # data starts `offset` elements in (misaligned base)
            keep.append(t)
            fx.fx_expr_bind(h, k, t.data_ptr() + offset * t.element_size(), b.rows, b.cols, b.ld)
        outs = {}
        rdt = torch.float64 if storage == "f64" else torch.float32
        if kind in ("elementwise", "multi"):
            ldz = R if ldz is None else ldz
            z = canary_buffer(max(ldz, 1) * C, torch_dtype(storage))
            fx.fx_expr_bind(h, n_in, z.data_ptr(), R, C, max(ldz, 1))
            outs["Z"] = (z, "z")
        if kind in ("full_reduce", "multi"):
            s = canary_buffer(1, rdt)
            fx.fx_expr_bind(h, n_in + (1 if kind == "multi" else 0), s.data_ptr(), 1, 1, 1)
            outs["s"] = (s, "s")
        if kind == "dim_reduce":
            d = 0 if name == "schur_colsum" else 1
            if d == 0:
                v = canary_buffer(C, rdt)
                fx.fx_expr_bind(h, n_in, v.data_ptr(), 1, C, 1)
            else:
                v = canary_buffer(R, rdt)
                fx.fx_expr_bind(h, n_in, v.data_ptr(), R, 1, max(R, 1))
            outs["v"] = (v, "v")
        sp = 0 if stream is None else stream
        if tune is not None:
            fx.fx_tune(h, tune, sp)
        if unfused:
            fx.fx_eval_unfused(h, sp)
        else:
            fx.fx_eval(h, sp)
        torch.cuda.synchronize()
        fx.fx_expr_sync_status(h, sp)   # no bounded wait gave up
        launches = fx.fx_expr_last_launches(h)
        result = {}
        for key, (t, kindk) in outs.items():
            if kindk == "z":
                ldzz = max(ldz, 1)
                check_canary(t, ldzz * C)
                full = from_device(t[: ldzz * C], storage)
                zz = full.reshape(C, ldzz).T[:R, :] if R * C else np.zeros((R, C))
                if ldzz > R and C > 0:   # padding rows untouched
                    pad = t[: ldzz * C].view(C, ldzz)[:, R:]
                    assert bool(torch.isnan(pad.float()).all()), "write into ld padding"
                result["Z"] = zz
            elif kindk == "s":
                check_canary(t, 1)
                result["s"] = from_device(t[:1], "f64")[0]
            else:
                nv = C if name == "schur_colsum" else R
                check_canary(t, nv)
                result["v"] = from_device(t[:nv], "f64")
        result["_launches"] = launches
        result["_shape"] = tuple(fx.fx_expr_launch_shape(h))
        return result
    finally:
        fx.fx_expr_destroy(h)


# ---------------------------------------------------------------- comparison

def gate_of(name, scalars=None):
    """"m" or "sigma": the scale the tree's results are held to."""
    return gate_scale(tree_of(name, scalars))


def _pick(v, sg, mg, scale, gate):
    if scale == "both":
        return (v, sg, mg)
    if scale == "sigma" or (scale == "gate" and gate == "sigma"):
        return (v, sg)
    return (v, mg)


def oracle_outputs(name, env, scalars=None, sample=None, scale="gate"):
    """Oracle values and their scale: full matrices, or at `sample` = (R, C)
    index arrays. scale: "gate" (the tree's gating scale), "sigma", "m", or
    "both" (triples value, sigma, m)."""
    tree = tree_of(name, scalars)
    gate = gate_scale(tree)
    need_s = scale in ("both", "sigma") or (scale == "gate" and gate == "sigma")
    need_m = scale in ("both", "m") or (scale == "gate" and gate == "m")

    def elementwise(t):
        if sample is None:
            v, sg = oracle.evaluate_sigma(t, env) if need_s else (oracle.evaluate(t, env), None)
            mg = oracle.evaluate_mag(t, env) if need_m else None
        else:
            v, sg = oracle.at_sigma(t, env, *sample) if need_s else (oracle.at(t, env, *sample), None)
            mg = oracle.at_mag(t, env, *sample) if need_m else None
        return v, sg, mg

    def reduction(t):
        v, sg = oracle.evaluate_sigma(t, env) if need_s else (oracle.evaluate(t, env), None)
        mg = oracle.evaluate_mag(t, env) if need_m else None
        return v, sg, mg

    if name in SIDE_SUM:
        res = {"Z": _pick(*elementwise(tree), scale, gate)}
        side = SIDE_SUM[name]
        sgate = gate_scale(side)
        need_s = scale in ("both", "sigma") or (scale == "gate" and sgate == "sigma")
        need_m = scale in ("both", "m") or (scale == "gate" and sgate == "m")
        v, sg, mg = reduction(side)
        res["s"] = _pick(v[0, 0], None if sg is None else sg[0, 0],
                         None if mg is None else mg[0, 0], scale, sgate)
        return res
    if name == "schur_trans_accu":
        res = {"Z": _pick(*elementwise(tree), scale, gate)}
        v, sg, mg = reduction(f"(accu {tree})")
        res["s"] = _pick(v[0, 0], None if sg is None else sg[0, 0],
                         None if mg is None else mg[0, 0], scale, gate)
        return res
    root = oracle.parse(tree)
    if root.op in oracle.REDUCTIONS:
        v, sg, mg = reduction(tree)
        if root.op in ("accu", "norm"):
            return {"s": _pick(v[0, 0], None if sg is None else sg[0, 0],
                               None if mg is None else mg[0, 0], scale, gate)}
        return {"v": _pick(v.ravel(), None if sg is None else sg.ravel(),
                           None if mg is None else mg.ravel(), scale, gate)}
    return {"Z": _pick(*elementwise(tree), scale, gate)}


# ---------------------------------------------------------------- full-size comparison

# (label, ErrorReport.as_dict()) of the full-size comparisons of this session,
# printed at the end of the pytest run (conftest.pytest_terminal_summary)
REPORTS = []


def record(label, rep):
    REPORTS.append((label, rep.as_dict()))

def _workers():
    import os
    return max(1, min(32, os.cpu_count() or 1))


def panel_report(name, storage, Z, env, scalars=None, both=False, budget=1 << 22):
    """Element-by-element comparison of a whole element-wise output Z (an
    R x C FP64 array) with the oracle, column panel by column panel on a
    thread pool (numpy releases the interpreter lock in its array loops).
    Returns an ErrorReport under the tree's gate scale (and, with `both`,
    the other scale as well)."""
    from concurrent.futures import ThreadPoolExecutor
    tree = tree_of(name, scalars)
    gate = gate_scale(tree)
    R, C = Z.shape
    w = max(1, budget // max(R, 1))
    panels = [(c0, min(C, c0 + w)) for c0 in range(0, C, w)]
    want_s = both or gate == "sigma"
    want_m = both or gate == "m"

    def one(p):
        c0, c1 = p
        rr, cc = np.arange(R)[:, None], np.arange(c0, c1)[None, :]
        if want_s:
            v, sg = oracle.at_sigma(tree, env, rr, cc)
        else:
            v, sg = oracle.at(tree, env, rr, cc), None
        mg = oracle.at_mag(tree, env, rr, cc) if want_m else None
        rep = ErrorReport(storage, tolerance(name, storage), gate)
        shape = (R, c1 - c0)
        rep.add(Z[:, c0:c1], np.broadcast_to(v, shape),
                None if sg is None else np.broadcast_to(sg, shape),
                None if mg is None else np.broadcast_to(mg, shape))
        return rep

    total = ErrorReport(storage, tolerance(name, storage), gate)
    with ThreadPoolExecutor(_workers()) as ex:
        for rep in ex.map(one, panels):
            total.merge(rep)
    return total
