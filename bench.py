"""Benchmark: fused evaluation of the 8192 x 8192 FP32 expression workload.

One step evaluates, on four 8192 x 8192 column-major FP32 matrices X, Y, W,
V drawn i.i.d. N(0, 1) (seed 1):
    Z      = X % Y + sqrt(abs(W)) / (1 + exp(-V))
    colsum = sum(X % Y, 0)
    rowmax = max(abs(X - Y), 1)
    nrm    = norm(X - Y, 2)
each as one fused kernel. The metric is the effective HBM bandwidth:
algorithmic bytes (every input element read once, every output written
once) per second. Inputs (256 MiB each) are larger than L2, so no flush is
needed between iterations.

--gpus N runs N independent replicas (one process per GPU, launched by
torch.distributed.run); value = bytes of all ranks / max elapsed time.
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused-expr effective HBM GB/s (% of GB300 peak) and speedup vs unfused per-op"
WORKLOAD = "X%Y+sqrt(abs(W))/(1+exp(-V)), sum(X%Y,0), max(abs(X-Y),1), norm(X-Y,2) at 8192x8192"

# DRAM traffic per launch of the dominant kernel from an ncu capture, valid
# only while the kernel source hashes to the recorded value.
TRAFFIC = {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("core.cuh", "expr.cuh", "plan.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2604_22242_gb300", "csrc", "fx", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def alg_bytes(R, C, es, rs):
    """Algorithmic bytes of one step: inputs read once, outputs written once."""
    N = R * C
    z = 5 * N * es                  # X, Y, W, V in; Z out
    colsum = 2 * N * es + C * rs
    rowmax = 2 * N * es + R * rs
    nrm = 2 * N * es + rs
    return {"Z": z, "colsum": colsum, "rowmax": rowmax, "nrm": nrm}


TREES = [("schur_sqrt_sigmoid", "Z"), ("schur_colsum", "colsum"), ("absdiff_rowmax", "rowmax"),
         ("diff_norm", "nrm")]
ORACLE_TREES = {
    "Z": "(+ (% X Y) (/ (sqrt (abs W)) (+ 1.0 (exp (neg V)))))",
    "colsum": "(sum (% X Y) 0)",
    "rowmax": "(max (abs (- X Y)) 1)",
    "nrm": "(norm (- X Y))",
}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def make_inputs(R, C, storage, seed=1):
    import synth
    return synth.operands(seed, [("X", R, C), ("Y", R, C), ("W", R, C), ("V", R, C)], storage,
                          "normal")


def cpu_oracle_time(R, C, cols, storage):
    """Oracle on the first `cols` columns of the workload: (seconds, bytes)."""
    import oracle
    env = make_inputs(R, cols, storage)
    es = 8 if storage == "f64" else 4
    b = alg_bytes(R, cols, es, es)
    t0 = time.perf_counter()
    for _, key in TREES:
        oracle.evaluate(ORACLE_TREES[key], env)
    return time.perf_counter() - t0, sum(b.values())


def run_reference(args, rank, world):
    """The FP64 CPU oracle timed on a bounded sample of the workload per step."""
    if rank != 0:
        return
    R = args.size
    cols = args.ref_cols
    for _ in range(args.warmup):
        cpu_oracle_time(R, cols, cols, args.dtype)
    tot_t, tot_b = 0.0, 0
    for _ in range(args.steps):
        t, b = cpu_oracle_time(R, cols, cols, args.dtype)
        tot_t += t
        tot_b += b
    v = tot_b / tot_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * tot_t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows": R, "cols": R, "sample_cols": cols,
                   "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{R}x{cols} column panel of each input per step, FP64 "
                                   "numpy tree walker, single thread"},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2604_22242_gb300 as fx

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    R = C = args.size
    storage = args.dtype
    code = {"f32": fx.FX_F32, "f64": fx.FX_F64}[storage]
    es = 8 if storage == "f64" else 4
    tdt = torch.float64 if storage == "f64" else torch.float32
    env = make_inputs(R, C, storage)
    host = {k: torch.from_numpy(v.data).pin_memory() for k, v in env.items()}
    d = {k: v.to(dev) for k, v in host.items()}
    Z = torch.empty(R * C, dtype=tdt, device=dev)
    outs = {"Z": Z, "colsum": torch.empty(C, dtype=tdt, device=dev),
            "rowmax": torch.empty(R, dtype=tdt, device=dev),
            "nrm": torch.empty(1, dtype=tdt, device=dev)}
    shapes = {"Z": (R, C, R), "colsum": (1, C, 1), "rowmax": (R, 1, R), "nrm": (1, 1, 1)}
    inputs = {"schur_sqrt_sigmoid": "XYWV", "schur_colsum": "XY", "absdiff_rowmax": "XY",
              "diff_norm": "XY"}
    stream = torch.cuda.Stream(device=dev)
    sp = int(stream.cuda_stream)
    ex = {}
    for name, key in TREES:
        h = fx.fx_expr_create(name, code)
        for k, s in enumerate(inputs[name]):
            fx.fx_expr_bind(h, k, d[s].data_ptr(), R, C, R)
        r, c, ld = shapes[key]
        fx.fx_expr_bind(h, len(inputs[name]), outs[key].data_ptr(), r, c, ld)
        if args.tune:
            fx.fx_tune(h, "search", sp)
        ex[key] = h
    torch.cuda.synchronize()
    bytes_ = alg_bytes(R, C, es, es)
    step_bytes = sum(bytes_.values())

    ev_z = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]

    def step(i=None, unfused=False):
        launches = 0
        for name, key in TREES:
            h = ex[key]
            if i is not None and key == "Z":
                ev_z[i][0].record(stream)
            (fx.fx_eval_unfused if unfused else fx.fx_eval)(h, sp)
            if i is not None and key == "Z":
                ev_z[i][1].record(stream)
            launches += fx.fx_expr_last_launches(h)
        return launches

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clk = Clocks(local)
        clk.start()
        time.sleep(0.3)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        launches = 0
        for i in range(args.steps):
            launches += step(i)
        t1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        if world > 1:
            dist.barrier()
        ms = t0.elapsed_time(t1)
        z_ms = statistics.mean(a.elapsed_time(b) for a, b in ev_z)

        # unfused baseline: same step, one kernel per operator
        uk = max(3, args.steps // 4)
        for _ in range(2):
            step(unfused=True)
        torch.cuda.synchronize()
        u0 = torch.cuda.Event(enable_timing=True)
        u1 = torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for _ in range(uk):
            step(unfused=True)
        u1.record(stream)
        torch.cuda.synchronize()
        ums = u0.elapsed_time(u1) / uk

        # end to end through the C ABI with host buffers: inputs copied in,
        # every output copied back, each step
        hz = torch.empty(R * C, dtype=tdt).pin_memory()
        hsmall = {k: torch.empty_like(outs[k], device="cpu").pin_memory()
                  for k in ("colsum", "rowmax", "nrm")}
        hin = [host[s].data_ptr() for s in "XYWV"]

        def e2e_step():
            fx.fx_eval_host(ex["Z"], hin, [hz.data_ptr()], sp)
            for _, key in TREES[1:]:
                fx.fx_eval(ex[key], sp)
                hsmall[key].copy_(outs[key], non_blocking=True)

        ek = max(3, args.steps // 4)
        e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ek):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1) / ek

    if world > 1:
        t = torch.tensor([ms, ums, ems], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ums, ems = (float(x) for x in t.tolist())
    if rank != 0:
        return
    for h in ex.values():
        fx.fx_expr_destroy(h)
    peak, peak_kind = measured_peaks()
    value = world * step_bytes * args.steps / (ms / 1e3) / 1e9
    z_gbs = bytes_["Z"] / (z_ms / 1e3) / 1e9
    khash = kernel_source_hash()
    tr = TRAFFIC.get(("Z", storage))
    traffic = tr["bytes"] if tr and tr["hash"] == khash else None

    cpu = None
    if world == 1 and not args.no_cpu:
        t_cpu, b_cpu = cpu_oracle_time(R, C, args.cpu_cols, storage)
        cpu = {"value": round(b_cpu / t_cpu / 1e9, 4), "unit": "GB/s", "cores": 1,
               "kind": "oracle",
               "sample": f"{R}x{args.cpu_cols} column panel of each input, all four trees, "
                         "FP64 numpy tree walker, single thread"}
    h2d = 4 * R * C * es
    d2h = R * C * es + (R + C + 1) * es
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": storage,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows": R, "cols": C, "layout": "column-major",
                   "inputs": "X,Y,W,V i.i.d. N(0,1), seed 1",
                   "l2": "inputs larger than L2 (256 MiB each), no flush",
                   "parallelism": f"replicas x{world}"},
        "pct_of_peak": round(100 * value / world / peak, 2),
        "pct_of_8tbs_spec": round(100 * value / world / 8000, 2),
        "vs_unfused": round(ums / (ms / args.steps), 3),
        "unfused_ms_per_step": round(ums, 4),
        "per_tree_bytes": bytes_,
        "roofline": {"bound": "hbm", "achieved": round(z_gbs, 2), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(z_gbs / peak, 4),
                     "traffic": traffic, "kernel": "k_flat (Z tree)",
                     "alg_bytes_per_launch": bytes_["Z"], "avg_launch_ms": round(z_ms, 4)},
        "e2e": {"value": round(world * step_bytes / (ems / 1e3) / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(ems, 3)},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--tune", action="store_true", help="autotune launch shapes first")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-cols", type=int, default=4096)
    ap.add_argument("--ref-cols", type=int, default=512)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world)
    finally:
        if world > 1 and args.impl == "ours":
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
