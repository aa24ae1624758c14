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


def _oracle_top(inst, k, s, seed, m, top):
    codes = O.encode(inst.ascii)
    h = O.hash_trials(codes, inst.seq_off, inst.l, k, s, seed, 0, m)
    sel = O.top_candidates(h["cand_cnt"], top)
    mem = [h["members"][h["cand_off"][c]:h["cand_off"][c + 1]] for c in sel]
    return h, sel, mem


@pytest.mark.parametrize("case", ["partitioned", "rehashed", "all_kept"])
def test_trial_hash_top_lists_bit_exact(P, chip_like, case):
    """The capped search's lists (Algorithm 2 step 3 with the top-K cap): which
    buckets are kept, in size order with (trial, key) ties, and every kept
    bucket's members in ascending order, bit for bit with the oracle.  The
    (20,5) t=200 input has x = 96,200 > 65,535 l-mers, so k = 10 takes the
    partitioned path (members gathered from the partition); a t=20 input at
    k = 7 rehashes each kept bucket's trial; a cap above C keeps everything."""
    if case == "partitioned":
        inst, k, s, m, top, seed = chip_like, 10, 3, 6, 64, 5
    elif case == "rehashed":
        from synth import instance_for_config
        inst, k, s, m, top, seed = instance_for_config(1), 7, 4, 30, 100, 11
    else:
        inst, k, s, m, top, seed = planted_instance(9, 1, 12, 300, 11, 2), 7, 4, 10, 10**5, 3
    packed = P.projection_pack(torch.from_numpy(inst.ascii).cuda())
    got = P.trial_hash_top(packed, inst.seq_off, inst.l, k, s, seed, m, top)
    h, sel, mem = _oracle_top(inst, k, s, seed, m, top)
    assert got["n_candidates"] == h["cand_key"].size
    assert got["n_members"] == h["members"].size
    assert got["n_kept"] == sel.size == min(top, h["cand_key"].size)
    if case != "all_kept":
        assert got["n_candidates"] > top
    assert np.array_equal(got["sel_index"].cpu().numpy(), sel)
    assert np.array_equal(got["cand_trial"].cpu().numpy(), h["cand_trial"][sel])
    assert np.array_equal(got["cand_key"].cpu().numpy().view(np.uint32),
                          h["cand_key"][sel].astype(np.uint32))
    assert np.array_equal(got["cand_cnt"].cpu().numpy(), h["cand_cnt"][sel])
    off = got["cand_off"].cpu().numpy()
    members = got["members"].cpu().numpy()
    assert off[0] == 0 and off[-1] == members.size == sum(len(v) for v in mem)
    for i, want in enumerate(mem):
        assert np.array_equal(members[off[i]:off[i + 1]], want), i


@pytest.mark.parametrize("prec,pwm_tol,ll_rel", [("fp32", 1e-5, 1e-6), ("bf16", 5e-5, 1e-4)])
def test_top_search_at_full_size(P, prec, pwm_tol, ll_rel):
    """The serving-scale input at full size (t = 2000 x n = 500, x = 962,000
    l-mers, k = 10), 3 trials, top 1024 buckets refined by 10 EM iterations.
    The oracle hashes the same trials; EM parity on the 16 largest buckets and
    the search's winner, from identical starting models (the oracle's theta^0
    rounded to float32): models and log-likelihoods within the precision's
    tolerance; the winner is one of the oracle's kept buckets, and its
    consensus and sites follow from its model."""
    from synth import instance_for_config
    inst = instance_for_config(5)
    k, s, m, top, iters = 10, 4, 3, 1024, 10
    precision = P.PROJ_EM_FP32 if prec == "fp32" else P.PROJ_EM_BF16_SPLIT
    packed = P.projection_pack(torch.from_numpy(inst.ascii).cuda())
    got = P.projection_find_packed_top(packed, inst.seq_off, inst.l, inst.d, k, s, m, seed=1005,
                                       em_iters=iters, pseudocount=0.25, precision=precision,
                                       top=top)
    codes = O.encode(inst.ascii)
    h = O.hash_trials(codes, inst.seq_off, inst.l, k, s, 1005, 0, m)
    kept = O.top_candidates(h["cand_cnt"], top)
    assert got["n_candidates"] == h["cand_key"].size and got["n_refined"] == top
    w = got["win_index"]
    assert w in set(kept.tolist())
    sel = list(kept[:16]) + ([w] if w not in set(kept[:16].tolist()) else [])
    th0 = np.stack([O.theta0(codes, inst.seq_off, inst.l,
                             h["members"][h["cand_off"][c]:h["cand_off"][c + 1]], 0.25)
                    for c in sel]).astype(np.float32)
    bg_o = O.background(codes)
    w_pwm, w_ll = O.em(codes, inst.seq_off, inst.l, bg_o, th0.astype(np.float64), iters, 0.25,
                       nthreads=16)
    bg = P.projection_background(packed, inst.seq_off[-1])
    g_pwm, g_ll = P.em_refine(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(),
                              iters, 0.25, precision)
    g_pwm, g_ll = g_pwm.cpu().numpy(), g_ll.cpu().numpy()
    assert np.max(np.abs(g_pwm - w_pwm)) <= pwm_tol
    assert np.all(np.abs(g_ll - w_ll) <= ll_tol(w_ll, inst.t, ll_rel))
    q = sel.index(w)
    assert np.max(np.abs(got["pwm"] - w_pwm[q])) <= pwm_tol
    assert abs(got["loglik"] - w_ll[q]) <= ll_tol(w_ll[q], inst.t, ll_rel)
    assert got["consensus"] == O.consensus(got["pwm"].astype(np.float64))
    assert np.array_equal(got["sites"], O.sites(codes, inst.seq_off, inst.l, bg_o,
                                                got["pwm"].astype(np.float64)))
