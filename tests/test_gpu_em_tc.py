"""Parity of the tensor-core EM path (PROJ_EM_BF16_SPLIT) with the FP64 oracle.

The log-odds matrix W and the posteriors P enter the MMAs as BF16 hi + lo
pairs: each entry keeps ~16 significant bits (|v - hi - lo| <= 2^-16 |v|).
The score error per l-mer is then bounded by 2^-16 sum_p |W_p| (log2 units)
plus FP32 accumulation, which for |W| <= ~5 and l <= 20 is a few 1e-5 typical
(1e-3 worst case with every sign aligned).  Tolerances used here, with ~3x
margin over the largest errors measured on the configs below: PWM entries
within 5e-5 absolute, log-likelihood ratios within 1e-4 relative (scale
floored at t nats).  The winner's consensus and sites must equal the oracle's
(equal motif recovery)."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import instance_for_config, planted_instance
from tests.conftest import ll_tol, oracle_theta0_sample

pytestmark = pytest.mark.gpu

PWM_TOL_BF16 = 5e-5
LL_REL_BF16 = 1e-4


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


def upload(P, ascii_bytes):
    return P.projection_pack(torch.from_numpy(np.frombuffer(bytes(ascii_bytes), np.uint8).copy())
                             .cuda())


def _theta0(P, inst, packed, k, s, seed, n, trials=20):
    return oracle_theta0_sample(inst, k, s, seed, n, trials)


CASES = {
    "cfg1": (lambda: instance_for_config(1), 7, 4, 300, 5),
    "cfg2": (lambda: instance_for_config(2), 7, 4, 260, 5),
    "cfg3": (lambda: instance_for_config(3), 8, 3, 129, 8),
    "l20_markov": (lambda: planted_instance(3, 0, 60, 500, 20, 5, background="markov_gc40"),
                   10, 4, 130, 10),
    "l6": (lambda: planted_instance(4, 0, 20, 300, 6, 1), 4, 4, 140, 5),
    "l32": (lambda: planted_instance(5, 0, 20, 300, 32, 8), 10, 2, 60, 5),
    "ragged": (lambda: planted_instance(77, 0, 13, [60, 500, 33, 900, 250, 17, 1200, 64, 400, 19,
                                                    700, 88, 301], 15, 3), 6, 3, 77, 5),
    "tiny_C": (lambda: instance_for_config(1), 7, 4, 3, 5),
}


@pytest.mark.parametrize("h", [2, 4])
@pytest.mark.parametrize("name", sorted(CASES))
def test_em_bf16_split_matches_oracle(P, name, h, monkeypatch):
    """Both kernel shapes: h = 2 (tiles of 64 l-mers, two CTAs per SM) and h = 4
    (tiles of 128 l-mers, four threads per candidate row, one CTA per SM)."""
    monkeypatch.setenv("PROJ_EM_SCHED", f"{2 if h == 2 else 1},1,{h}")
    make, k, s, n, iters = CASES[name]
    inst = make()
    codes = O.encode(inst.ascii)
    packed = upload(P, inst.ascii)
    th0 = _theta0(P, inst, packed, k, s, 7, n)
    bg = P.projection_background(packed, inst.seq_off[-1])
    pwm, ll = P.em_refine(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(), iters,
                          0.25, P.PROJ_EM_BF16_SPLIT)
    w_pwm, w_ll = O.em(codes, inst.seq_off, inst.l, O.background(codes), th0.astype(np.float64),
                       iters, 0.25, nthreads=16)
    pwm, ll = pwm.cpu().numpy(), ll.cpu().numpy()
    assert np.max(np.abs(pwm - w_pwm)) <= PWM_TOL_BF16
    assert np.all(np.abs(ll - w_ll) <= ll_tol(w_ll, inst.t, LL_REL_BF16))
    assert np.allclose(pwm.sum(axis=2), 1.0, atol=1e-5)


def test_em_bf16_split_estep_only(P):
    inst = instance_for_config(2)
    codes = O.encode(inst.ascii)
    packed = upload(P, inst.ascii)
    th0 = _theta0(P, inst, packed, 7, 4, 9, 200)
    bg = P.projection_background(packed, inst.seq_off[-1])
    pwm, ll = P.em_refine(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(), 0, 0.25,
                          P.PROJ_EM_BF16_SPLIT)
    _, w_ll = O.em(codes, inst.seq_off, inst.l, O.background(codes), th0.astype(np.float64), 0,
                   0.25, nthreads=16)
    assert np.array_equal(pwm.cpu().numpy(), th0)  # no M-step: the model is unchanged
    assert np.all(np.abs(ll.cpu().numpy() - w_ll) <= ll_tol(w_ll, inst.t, LL_REL_BF16))


def test_em_bf16_split_is_deterministic(P):
    inst = instance_for_config(1)
    packed = upload(P, inst.ascii)
    th0 = torch.from_numpy(_theta0(P, inst, packed, 7, 4, 3, 500)).cuda()
    bg = P.projection_background(packed, inst.seq_off[-1])
    a = P.em_refine(packed, inst.seq_off, inst.l, bg, th0, 5, 0.25, P.PROJ_EM_BF16_SPLIT)
    b = P.em_refine(packed, inst.seq_off, inst.l, bg, th0, 5, 0.25, P.PROJ_EM_BF16_SPLIT)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("cfg", [1, 2])
def test_find_bf16_split_recovers_the_oracle_motif(P, cfg):
    inst = instance_for_config(cfg)
    prm = inst.params
    got = P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, prm["k"], prm["s"],
                            prm["m"], seed=1000 + cfg, em_iters=prm["em_iters"],
                            pseudocount=prm["beta"], precision=P.PROJ_EM_BF16_SPLIT)
    want = O.find([q.decode() for q in inst.seqs], inst.l, inst.d, prm["k"], prm["s"], prm["m"],
                  seed=1000 + cfg, em_iters=prm["em_iters"], beta=prm["beta"], nthreads=16)
    assert got["n_candidates"] == want["n_candidates"]
    assert got["consensus"] == want["consensus"]
    assert np.array_equal(got["sites"], want["sites"])
    assert abs(got["loglik"] - want["loglik"]) <= ll_tol(want["loglik"], inst.t, LL_REL_BF16)
    fp32 = P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, prm["k"], prm["s"],
                             prm["m"], seed=1000 + cfg, em_iters=prm["em_iters"],
                             pseudocount=prm["beta"], precision=P.PROJ_EM_FP32)
    assert fp32["consensus"] == got["consensus"] and np.array_equal(fp32["sites"], got["sites"])


def _peaked_models(rng, inst, n_peaked, n_flat, hi=0.997):
    """n_peaked models putting `hi` on one base per column (the bases of
    planted-motif-like l-mers), then n_flat models near uniform."""
    l = inst.l
    th = np.empty((n_peaked + n_flat, l, 4), np.float64)
    motif = O.encode(inst.motif.encode())
    for c in range(n_peaked):
        word = motif.copy()
        flip = rng.choice(l, size=int(rng.integers(0, 4)), replace=False)
        word[flip] = rng.integers(0, 4, flip.size)
        th[c] = (1.0 - hi) / 3.0
        th[c, np.arange(l), word] = hi
    th[n_peaked:] = rng.dirichlet(np.full(4, 20.0), size=(n_flat, l))
    return th.astype(np.float32)


@pytest.mark.parametrize("h", [2, 4])
def test_em_bf16_split_careful_rows(P, h, monkeypatch):
    """Rows whose score range sum_p (max_a W - min_a W) exceeds 200 (log2 units)
    switch their CTA to careful mode: exact first-tile maxima and a per-tile
    overflow check with rescaling.  Peaked models (0.997 / 0.001 per column,
    l = 24: range ~240) exercise it; the second candidate tile holds only flat
    models and stays in fast mode in the same launch.  Measured errors: PWM
    2.5e-6, LL 5.8e-5 relative (E-step only); the LL tolerance is doubled over
    the planted-workload one for a ~3x margin (the BF16-split score error bound
    2^-16 sum_p |W_p| grows with the range).  A wrong rescale would be off by
    powers of two or non-finite."""
    monkeypatch.setenv("PROJ_EM_SCHED", f"{2 if h == 2 else 1},1,{h}")
    inst = planted_instance(21, 0, 20, 400, 24, 4)
    rng = np.random.default_rng(5)
    th0 = _peaked_models(rng, inst, 100, 60)
    codes = O.encode(inst.ascii)
    packed = upload(P, inst.ascii)
    bg = P.projection_background(packed, inst.seq_off[-1])
    for iters in (0, 4):
        pwm, ll = P.em_refine(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(), iters,
                              0.25, P.PROJ_EM_BF16_SPLIT)
        w_pwm, w_ll = O.em(codes, inst.seq_off, inst.l, O.background(codes),
                           th0.astype(np.float64), iters, 0.25, nthreads=16)
        pwm, ll = pwm.cpu().numpy(), ll.cpu().numpy()
        assert np.all(np.isfinite(pwm)) and np.all(np.isfinite(ll))
        assert np.max(np.abs(pwm - w_pwm)) <= PWM_TOL_BF16
        assert np.all(np.abs(ll - w_ll) <= ll_tol(w_ll, inst.t, 2 * LL_REL_BF16))
