"""ZOOPS EM on the GPU (zero or one site per sequence, fixed site probability;
reading R15) against the FP64 oracle's statement of the same model: both
precision paths from identical starting models, the site_prob = 1 reduction to
the OOPS path, and a whole top-K search on a ZOOPS-planted input."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import planted_instance
from tests.conftest import ll_tol, oracle_theta0_sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


def _upload(P, inst):
    return P.projection_pack(torch.from_numpy(np.frombuffer(bytes(inst.ascii), np.uint8).copy())
                             .cuda())


@pytest.fixture(scope="module")
def case():
    inst = planted_instance(31, 0, 40, 400, 15, 4, zoops_frac=0.6)
    th0 = oracle_theta0_sample(inst, 7, 4, 5, 300, 6)
    return inst, th0


@pytest.mark.parametrize("gamma", [0.6, 0.25])
@pytest.mark.parametrize("prec,pwm_tol,ll_rel", [("fp32", 1e-5, 1e-6), ("bf16", 5e-5, 1e-4)])
def test_zoops_em_matches_oracle(P, case, gamma, prec, pwm_tol, ll_rel):
    inst, th0 = case
    codes = O.encode(inst.ascii)
    want_th, want_ll = O.em_zoops(codes, inst.seq_off, inst.l, O.background(codes),
                                  th0.astype(np.float64), 5, 0.25, gamma, nthreads=16)
    packed = _upload(P, inst)
    bg = P.projection_background(packed, inst.seq_off[-1])
    precision = P.PROJ_EM_FP32 if prec == "fp32" else P.PROJ_EM_BF16_SPLIT
    th, ll = P.em_refine_zoops(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(), 5,
                               0.25, gamma, precision)
    th, ll = th.cpu().numpy(), ll.cpu().numpy()
    assert np.max(np.abs(th - want_th)) <= pwm_tol
    assert np.all(np.abs(ll - want_ll) <= ll_tol(want_ll, inst.t, ll_rel))
    assert np.allclose(th.sum(axis=2), 1.0, atol=1e-5)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_zoops_gamma_one_is_oops(P, case, prec):
    inst, th0 = case
    packed = _upload(P, inst)
    bg = P.projection_background(packed, inst.seq_off[-1])
    precision = P.PROJ_EM_FP32 if prec == "fp32" else P.PROJ_EM_BF16_SPLIT
    t0 = torch.from_numpy(th0).cuda()
    a = P.em_refine(packed, inst.seq_off, inst.l, bg, t0, 4, 0.25, precision)
    b = P.em_refine_zoops(packed, inst.seq_off, inst.l, bg, t0, 4, 0.25, 1.0, precision)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_zoops_rejects_bad_site_probability(P, case):
    inst, th0 = case
    packed = _upload(P, inst)
    bg = P.projection_background(packed, inst.seq_off[-1])
    for g in (0.0, 1.5):
        with pytest.raises(P.ProjectionError):
            P.em_refine_zoops(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(), 2,
                              0.25, g)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_zoops_search_matches_oracle(P, case, prec):
    """Whole search with top-K refinement under ZOOPS: the winner's consensus
    and sites and its log-likelihood against the oracle (hash, top-K choice,
    theta^0, ZOOPS EM, FP64 ranking, sites, all on the CPU)."""
    inst, _ = case
    k, s, m, top, gamma = 7, 4, 12, 256, 0.6
    codes = O.encode(inst.ascii)
    h = O.hash_trials(codes, inst.seq_off, inst.l, k, s, 77, 0, m)
    sel = O.top_candidates(h["cand_cnt"], top)
    th0 = np.stack([O.theta0(codes, inst.seq_off, inst.l,
                             h["members"][h["cand_off"][c]:h["cand_off"][c + 1]], 0.25) for c in sel])
    bg = O.background(codes)
    pwm, ll = O.em_zoops(codes, inst.seq_off, inst.l, bg, th0, 5, 0.25, gamma, nthreads=16)
    b = O.rank(ll)
    want_sites = O.sites(codes, inst.seq_off, inst.l, bg, pwm[b])
    precision = P.PROJ_EM_FP32 if prec == "fp32" else P.PROJ_EM_BF16_SPLIT
    got = P.projection_find_packed_zoops(_upload(P, inst), inst.seq_off, inst.l, inst.d, k, s, m,
                                         seed=77, em_iters=5, pseudocount=0.25,
                                         precision=precision, site_prob=gamma, top=top)
    assert got["n_candidates"] == h["cand_key"].size and got["n_refined"] == sel.size
    rel = 1e-6 if prec == "fp32" else 1e-4
    assert abs(got["loglik"] - ll[b]) <= ll_tol(ll[b], inst.t, rel)
    if got["win_index"] != int(sel[b]):
        # a tie within the tolerance: the GPU's winner must be a near-best model
        j = int(np.nonzero(sel == got["win_index"])[0][0])
        assert abs(ll[j] - ll[b]) <= ll_tol(ll[b], inst.t, rel)
    else:
        assert got["consensus"] == O.consensus(pwm[b])
        assert np.array_equal(got["sites"], want_sites)
