"""Low-memory enrichment by all-pairs comparison (PROJECTION2 / Section 6's
pairwise compare): its candidate and member lists must equal the oracle's and
the histogram path's bit for bit (integer work)."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import instance_for_config, planted_instance
from tests.test_gpu_parity import assert_hash_equal, hash_np, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


@pytest.mark.parametrize("cfg,trials", [(1, 8), (2, 6)])
def test_allpairs_matches_oracle(P, cfg, trials):
    inst = instance_for_config(cfg)
    prm = inst.params
    codes = O.encode(inst.ascii)
    want = O.hash_trials(codes, inst.seq_off, inst.l, prm["k"], prm["s"], 1000 + cfg, 3, 3 + trials)
    h = P.trial_hash_allpairs(upload(P, inst.ascii), inst.seq_off, inst.l, prm["k"], prm["s"],
                              1000 + cfg, 3, trials)
    assert_hash_equal(hash_np(h), want)


@pytest.mark.parametrize("seed", range(3))
def test_allpairs_ragged_small_and_histogram_path(P, seed):
    rng = np.random.default_rng(seed)
    lens = [int(v) for v in rng.integers(9, 300, 11)]
    inst = planted_instance(60 + seed, 0, 11, lens, 9, 2)
    packed = upload(P, inst.ascii)
    k, s = int(rng.integers(3, 8)), int(rng.integers(2, 5))
    a = P.trial_hash_allpairs(packed, inst.seq_off, 9, k, s, seed, 0, 5)
    b = P.trial_hash(packed, inst.seq_off, 9, k, s, seed, 0, 5)
    assert_hash_equal(hash_np(a), hash_np(b))
    codes = O.encode(inst.ascii)
    assert_hash_equal(hash_np(a), O.hash_trials(codes, inst.seq_off, 9, k, s, seed, 0, 5))


def test_allpairs_rejects_large_k(P):
    inst = instance_for_config(1)
    with pytest.raises(P.ProjectionError):
        P.trial_hash_allpairs(upload(P, inst.ascii), inst.seq_off, 11, 16, 3, 0, 0, 1)
