"""The autotuner (GPU): a search times every candidate launch shape and
kernel variant on the bound buffers, keeps the fastest, records it in the
cache file, and a later object of the same tree, storage and shape class
picks it up from the cache; results stay within tolerance either way."""
import json

import pytest

import synth
from harness import oracle_outputs, run, scaled_error, specs_for, tolerance

pytestmark = pytest.mark.gpu

BLOCKS, UNROLLS, BPS, PIPES = {128, 256, 512}, {2, 4, 8}, {0, 2, 4}, {0, 1, 2}


@pytest.fixture(scope="module")
def fx(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fxlib


@pytest.mark.parametrize("name", ["schur_exp_trans", "sqdiff_accu", "absdiff_rowmax"])
def test_search_then_cache(fx, name, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("FX_TUNE_CACHE", str(cache))
    R, C = 520, 384
    env = synth.operands(120, specs_for(name, R, C), "f32", "uniform")
    ref = oracle_outputs(name, env)
    got = run(fx, name, "f32", env, R, C, tune="search")
    b, u, s, p = got["_shape"]
    assert b in BLOCKS and u in UNROLLS and s in BPS and p in PIPES
    for key, (rv, rs) in ref.items():
        err, _, bad, _ = scaled_error(got[key], rv, rs, "f32")
        assert bad == 0 and err <= tolerance(name, "f32", key)
    entries = json.loads(cache.read_text())
    assert len(entries) == 1
    assert list(entries.values())[0] == f"{b},{u},{s},{p}"
    again = run(fx, name, "f32", env, R, C, tune="cache")
    assert again["_shape"] == (b, u, s, p)
    off = run(fx, name, "f32", env, R, C, tune="off")
    assert off["_shape"] == (256, 4, 0, 0)
