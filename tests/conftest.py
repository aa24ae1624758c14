import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: runs for more than a few seconds")


def golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


@pytest.fixture(scope="session")
def fig1():
    """Figure 1's seven sequences as a list of str."""
    return golden_lines("fig1_sequences.txt")


@pytest.fixture(scope="session")
def native_lib():
    """The CUDA library, built for sm_103a if it is missing or stale."""
    from paper_1605_06904_gb300 import _build, _native
    _build.build()
    return _native.lib()


def ll_tol(want, t, rel=1e-6):
    """Tolerance on a log-likelihood ratio: `rel` relative, with the scale
    floored at t (one nat per sequence; LL is a sum of t per-sequence terms
    each rounded at FP32 precision)."""
    import numpy as np
    return rel * np.maximum(np.abs(want), t)
