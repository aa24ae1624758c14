"""Refining only the largest enriched buckets (projection_find_top), as the
serving-scale workload does (top 1024 of ~10^7): the selection must equal the
oracle's (size descending, ties in (trial, key) order), and the motif, sites
and scores must match the oracle in both EM precisions."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import planted_instance
from tests.conftest import ll_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


@pytest.fixture(scope="module")
def chip_like():
    """Config-5 shape at reduced size: Markov background with 40% GC, (20,5)
    planted in 60% of the sequences."""
    return planted_instance(1005, 7, 200, 500, 20, 5, background="markov_gc40", zoops_frac=0.6)


@pytest.mark.parametrize("prec,pwm_tol,ll_rel", [("fp32", 1e-5, 1e-6), ("bf16", 5e-5, 1e-4)])
def test_top_refinement_matches_oracle(P, chip_like, prec, pwm_tol, ll_rel):
    inst = chip_like
    k, s, m, top, iters = 10, 3, 8, 64, 10
    precision = P.PROJ_EM_FP32 if prec == "fp32" else P.PROJ_EM_BF16_SPLIT
    got = P.projection_find_top(inst.ascii, inst.seq_off, 20, 5, k, s, m, seed=5, em_iters=iters,
                                pseudocount=0.25, precision=precision, top=top)
    want = O.find([q.decode() for q in inst.seqs], 20, 5, k, s, m, seed=5, em_iters=iters,
                  beta=0.25, nthreads=16, top=top, with_hash=True)
    assert got["n_candidates"] == want["n_candidates"] > top
    assert got["n_refined"] == top
    # the winner indexes the full list and is one of the oracle's selected buckets
    assert got["win_index"] in set(want["cand_index"].tolist())
    assert got["consensus"] == want["consensus"]
    assert np.array_equal(got["sites"], want["sites"])
    assert abs(got["loglik"] - want["loglik"]) <= ll_tol(want["loglik"], inst.t, ll_rel)
    assert np.max(np.abs(got["pwm"] - want["pwm"])) <= pwm_tol
    h = want["hash"]
    assert got["win_trial"] == h["cand_trial"][got["win_index"]]
    assert got["win_key"] == h["cand_key"][got["win_index"]]


def test_top_larger_than_candidates_refines_all(P):
    inst = planted_instance(9, 1, 12, 300, 11, 2)
    a = P.projection_find_top(inst.ascii, inst.seq_off, 11, 2, 7, 4, 10, seed=3, em_iters=3,
                              top=10**6)
    b = P.projection_find(inst.ascii, inst.seq_off, 11, 2, 7, 4, 10, seed=3, em_iters=3)
    assert a["n_refined"] == a["n_candidates"] == b["n_candidates"]
    for key in ("win_index", "consensus", "loglik", "score"):
        assert a[key] == b[key]
    assert np.array_equal(a["sites"], b["sites"])
