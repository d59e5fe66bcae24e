"""Host logic of bench.py on CPU: the replica path with two ranks (gloo),
where the slowest rank's time sets the whole-job number and only rank 0
reports, and the lookup of the recorded DRAM traffic."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.aggregate(10.0 + rank, 2.0e9, 4, world, dist)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, value))


def test_aggregate_takes_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 11.0                                   # the slower rank
        assert value == pytest.approx(2 * 2.0e9 * 4 / 0.011 / 1e9)


def test_reference_arm_reports_on_rank0_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-cols", "8"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""
    env["RANK"] = "0"
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-cols", "8"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_recorded_traffic_matches_source_and_shape():
    """The dominant kernel's DRAM traffic is reported only for the kernel
    sources and launch shapes it was captured at."""
    import bench
    h = bench.kernel_source_hash()
    tr = bench.TRAFFIC[("expr8192", "Z")]
    (block, unroll), nbytes = next(iter(tr["bytes"].items()))
    if tr["hash"] == h:
        assert bench.recorded_traffic("expr8192", "Z", (block, unroll, 0, 0), h) == nbytes
        assert bench.recorded_traffic("expr8192", "Z", (block, unroll, 4, 2), h) == nbytes
    assert bench.recorded_traffic("expr8192", "Z", (block, unroll, 0, 0), "0" * 16) is None
    assert bench.recorded_traffic("expr8192", "Z", (block, unroll, 0, 1), tr["hash"]) is None
    assert bench.recorded_traffic("expr8192", "Z", (96, 16, 0, 0), tr["hash"]) is None
    assert bench.recorded_traffic("suite10k", "add16", (256, 4, 0, 0), tr["hash"]) is None
    # every recorded figure is the same streaming pass: algorithmic reads plus
    # at most the algorithmic writes
    alg_read, alg_write = 4 * 8192 * 8192 * 4, 8192 * 8192 * 4
    for b in tr["bytes"].values():
        assert alg_read <= b <= alg_read * 1.001 + alg_write


def test_oracle_check_leg_on_cpu_tensors():
    """bench.oracle_errors on outputs held in CPU tensors: the oracle's own
    values rounded to the storage type pass, and a planted error fails."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    R, C = 64, 48
    env = synth.operands(1, [("X", R, C), ("Y", R, C), ("W", R, C), ("V", R, C)], "f32", "normal")
    keep = {"env": env, "trees": []}
    for name, key, ins, kind in [("schur_sqrt_sigmoid", "Z", "XYWV", "Z"),
                                 ("schur_colsum", "colsum", "XY", "col"),
                                 ("absdiff_rowmax", "rowmax", "XY", "row"),
                                 ("diff_norm", "nrm", "XY", "s")]:
        v = oracle.evaluate(bench.ORACLE_OF[name], env)
        flat = v.T.ravel() if kind == "Z" else v.ravel()
        keep[key] = (None, torch.from_numpy(flat.astype(np.float32)))
        keep["trees"].append((name, key, list(ins), kind))
    errs = bench.oracle_errors(keep, "f32", n_sample=512)
    assert set(errs) == {"Z", "colsum", "rowmax", "nrm"}
    for k, d in errs.items():
        assert d["ok"], (k, d)
        assert d["gate"] == ("sigma" if k == "Z" else "m")
        assert d["max_scaled_err_sigma"] is not None and d["max_scaled_err_m"] is not None
    keep["colsum"][1][3] += 0.01 * float(keep["colsum"][1].abs().max())
    assert not bench.oracle_errors(keep, "f32", n_sample=512)["colsum"]["ok"]


def test_oracle_check_leg_maps_suite_operands_to_slots():
    """The Sec. 4 suite binds operands named A1.., P1, Y64 to trees whose
    slots are X, Y, A, B ...: bench.oracle_errors must evaluate each tree on
    its own slot names. Outputs made from the test harness's trees (typed
    separately from the bench's) pass; a planted error in one fails."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    from tests import harness
    R = C = 40
    env = synth.operands(4, [(f"A{k}", R, C) for k in range(1, 6)], "f32", "uniform")
    env.update(synth.operands(5, [("P1", R, C), ("P2", R, C)], "f32", "positive"))
    env.update(synth.operands(6, [("Y64", R, C)], "f64", "normal"))
    trees = [("add5", "add5", [f"A{k}" for k in range(1, 6)]),
             ("expr1", "expr1", ["A1", "A2"]), ("expr2", "expr2", ["A1", "A2", "A3", "A4"]),
             ("expr3", "expr3", ["P1", "Y64", "P2"]), ("relu", "relu", ["A1"]),
             ("sigmoid", "sigmoid", ["A1"]), ("swish", "swish", ["A1"]), ("gelu", "gelu", ["A1"])]
    keep = {"env": env, "trees": []}
    for name, key, ins in trees:
        senv = {slot: env[i] for slot, i in zip(harness.SLOTS[name], ins)}
        v = oracle.evaluate(harness.tree_of(name), senv)
        keep[key] = (None, torch.from_numpy(v.T.ravel().astype(np.float32)))
        keep["trees"].append((name, key, ins, "Z"))
    errs = bench.oracle_errors(keep, "f32", n_sample=256)
    assert set(errs) == {k for _, k, _ in trees}
    for k, d in errs.items():
        assert d["ok"], (k, d)
    z = keep["gelu"][1]
    z += 1e-3 * float(z.abs().max())
    assert not bench.oracle_errors(keep, "f32", n_sample=256)["gelu"]["ok"]
