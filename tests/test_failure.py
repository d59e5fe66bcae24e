"""Failure detection without a GPU fault.

On the GPU: a bounded wait that nothing releases gives up, records the
timeout in the error word, and the kernel finishes (the path every
TMA / bulk / cp.async pipeline takes when a copy never lands); the context
stays usable afterwards. On the host: injected launch and allocation
failures come back as status codes (tests/test_capi.py covers the host
checks without a GPU).
"""
import os
import subprocess
import sys

import pytest


@pytest.mark.gpu
def test_bounded_wait_gives_up(fxlib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert fxlib.fx_selftest_wait_timeout(0) == 1
    # the context still works: a normal evaluation afterwards
    x = torch.ones(64, device="cuda")
    assert float(x.sum()) == 64.0
    assert fxlib.fx_selftest_wait_timeout(0) == 1


@pytest.mark.gpu
@pytest.mark.parametrize("mode,status", [("launch_fail", -7), ("alloc_fail", -8)])
def test_injected_failures_on_device(mode, status):
    """FX_INJECT turns a launch or a workspace allocation into a reported
    failure (a child process, so the injection stays out of this one)."""
    code = (
        "import sys; sys.path.insert(0, '.'); sys.path.insert(0, 'tests')\n"
        "import torch, synth, paper_2604_22242_gb300 as fx\n"
        "from harness import run\n"
        "env = synth.operands(1, [('A', 64, 48), ('B', 64, 48)], 'f32', 'uniform')\n"
        "try:\n"
        "    run(fx, 'sqdiff_accu', 'f32', env, 64, 48)\n"
        "    print('no error')\n"
        "except fx.FxError as e:\n"
        "    print('status', e.status)\n")
    env = dict(os.environ, FX_INJECT=mode)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert f"status {status}" in out.stdout, out.stdout + out.stderr[-2000:]
