import os
import sys

import numpy as np
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
    floored at t nats.  LL = sum_i L_i over t sequences, each L_i computed in
    FP32 (max + log2 of a sum of ~10^2-10^3 exponentials) with an absolute error
    of about rel * max(1, |L_i|), so the sum's error is bounded by
    rel * sum_i max(1, |L_i|) >= rel * t, whatever |LL| is (the L_i can have
    either sign and cancel).  A floor of one nat instead fails FP32 parity at
    1e-6 on candidates with |LL| < t (measured: 10 cases in the GPU suite)."""
    import numpy as np
    return rel * np.maximum(np.abs(want), t)


def oracle_theta0_sample(inst, k, s, seed, n, trials, beta=0.25):
    """theta^0 of up to n evenly spaced candidates of `trials` trials, built by
    the oracle alone (hash, enrichment and Section 5.1's starting model) and
    rounded to float32: the shared input of EM parity tests."""
    import oracle as O
    codes = O.encode(inst.ascii)
    h = O.hash_trials(codes, inst.seq_off, inst.l, k, s, seed, 0, trials)
    C = h["cand_key"].size
    idx = np.unique(np.linspace(0, C - 1, min(n, C)).astype(np.int64))
    th = np.stack([O.theta0(codes, inst.seq_off, inst.l,
                            h["members"][h["cand_off"][c]:h["cand_off"][c + 1]], beta) for c in idx])
    return th.astype(np.float32)
