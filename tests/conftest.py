import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: full-size case (minutes of CPU oracle time)")


@pytest.fixture(scope="session")
def fxlib():
    """The built library (built here if missing; nvcc cross-compiles without a GPU)."""
    import paper_2604_22242_gb300 as fx
    from paper_2604_22242_gb300 import build as fxbuild
    fxbuild.build()
    fx.lib()
    return fx


def pytest_terminal_summary(terminalreporter):
    """Errors of the full-size comparisons against the oracle, one line each."""
    try:
        import harness
    except ImportError:
        return
    if not harness.REPORTS:
        return
    tr = terminalreporter
    tr.section("errors against the FP64 oracle (full-size outputs, every element)")
    for label, d in harness.REPORTS:
        def f(x):
            return "-" if x is None else f"{x:.2e}"
        tr.write_line(f"{label}: gate {d['gate']} err_sigma {f(d['max_scaled_err_sigma'])} "
                      f"err_m {f(d['max_scaled_err_m'])} rel {d['max_plain_rel_err']:.2e} "
                      f"tol {d['tol']:.0e} overflow {d['overflow_expected']} "
                      f"nonfinite {d['nonfinite']} n {d['compared']}")
