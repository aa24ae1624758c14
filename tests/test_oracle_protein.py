"""Pins of the oracle's protein-alphabet functions (reading R17: 20 letters,
keys base 20): with 4 letters they must reproduce the DNA functions exactly
(codes 0..3, keys base 4); bucket membership against an all-pairs brute force;
the one-l-mer-per-sequence EM closed form; the non-decreasing MAP objective;
and planted-motif recovery on an easy protein instance."""
import math

import numpy as np
import pytest

import oracle as O
from synth import planted_instance, planted_protein


def test_encode_aa_letters_and_rejects_others():
    assert O.encode_aa(b"ACDEFGHIKLMNPQRSTVWY").tolist() == list(range(20))
    assert O.encode_aa(b"wyc").tolist() == [18, 19, 1]
    with pytest.raises(ValueError):
        O.encode_aa(b"ACDB")


def test_alphabet_four_reproduces_the_dna_functions():
    inst = planted_instance(9, 0, 6, 80, 8, 1)
    codes = O.encode(inst.ascii)
    off = inst.seq_off
    pos = O.positions(3, 1, 8, 5)
    assert np.array_equal(O.keys_a(codes, off, 8, pos, 4), O.keys(codes, off, 8, pos))
    assert np.allclose(O.background_a(codes, 4), O.background(codes), rtol=0, atol=0)
    mem = np.array([0, 7, 40, 100], np.int32)
    assert np.array_equal(O.theta0_a(codes, off, 8, mem, 0.25, 4), O.theta0(codes, off, 8, mem, 0.25))
    pwm0 = O.theta0(codes, off, 8, mem, 0.25)[None]
    bg = O.background(codes)
    a = O.em(codes, off, 8, bg, pwm0, 3, 0.25)
    b = O.em_a(codes, off, 8, bg, pwm0, 3, 0.25, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(O.sites_a(codes, off, 8, bg, a[0][0], 4), O.sites(codes, off, 8, bg, a[0][0]))
    assert O.consensus_a(a[0][0], 4, "ACTG") == O.consensus(a[0][0])


@pytest.mark.parametrize("seed", range(3))
def test_protein_buckets_match_all_pairs(seed):
    rng = np.random.default_rng(seed)
    l, k = 6, int(rng.integers(1, 4))
    seqs = ["".join(O.AA_LETTERS[c] for c in rng.integers(0, 3, n)) for n in rng.integers(6, 25, 5)]
    codes = O.encode_aa("".join(seqs).encode())
    off = np.concatenate([[0], np.cumsum([len(q) for q in seqs])]).astype(np.int64)
    pos = np.sort(rng.choice(l, k, replace=False)).astype(np.int32)
    keys = O.keys_a(codes, off, l, pos, 20)
    lmers = [q[j:j + l] for q in seqs for j in range(len(q) - l + 1)]
    proj = ["".join(w[p] for p in pos) for w in lmers]
    for s in (1, 2, 3):
        ck, cc, co, mem = O.enriched(keys, s)
        got = {tuple(mem[co[c]:co[c + 1]].tolist()) for c in range(ck.size)}
        want = {tuple(h for h in range(len(proj)) if proj[h] == proj[g]) for g in range(len(proj))}
        assert got == {w for w in want if len(w) >= s}
    # key = base-20 number of the projected letters, first position most significant
    for g, w in enumerate(proj):
        assert keys[g] == sum(O.AA_LETTERS.index(ch) * 20 ** (len(w) - 1 - q) for q, ch in enumerate(w))


def test_protein_em_closed_form_and_monotone():
    rng = np.random.default_rng(4)
    l, beta = 5, 0.1
    seqs = ["".join(O.AA_LETTERS[c] for c in rng.integers(0, 20, l)) for _ in range(9)]
    codes = O.encode_aa("".join(seqs).encode())
    off = np.concatenate([[0], np.cumsum([l] * 9)]).astype(np.int64)
    bg = O.background_a(codes, 20)
    p0 = rng.random((l, 20)) + 0.05
    p0 /= p0.sum(axis=1, keepdims=True)
    pwm1, _ = O.em_a(codes, off, l, bg, p0[None], 1, beta, 20)
    cnt = np.zeros((l, 20))
    for q in seqs:
        for p, ch in enumerate(q):
            cnt[p, O.AA_LETTERS.index(ch)] += 1
    assert np.allclose(pwm1[0], (cnt + beta) / (9 + 20 * beta), rtol=0, atol=1e-14)
    inst = planted_protein(5, 0, 8, 60, 6, 1)
    codes = O.encode_aa(inst.ascii)
    bg = O.background_a(codes, 20)
    pwm = p0[:5].copy()
    pwm = np.vstack([pwm, pwm[:1]])
    prev = -np.inf
    for _ in range(8):
        ll = O.em_a(codes, inst.seq_off, 6, bg, pwm[None], 0, beta, 20)[1][0]
        obj = ll + beta * np.log(pwm).sum()
        assert obj >= prev - 1e-9 * max(1.0, abs(prev))
        prev = obj
        pwm = O.em_a(codes, inst.seq_off, 6, bg, pwm[None], 1, beta, 20)[0][0]
        assert np.allclose(pwm.sum(axis=1), 1.0, atol=1e-12)


def test_protein_planted_recovery():
    inst = planted_protein(7, 0, 15, 200, 10, 2)
    res = O.find_protein([q.decode() for q in inst.seqs], 10, 4, 3, 30, 1, 5, 0.1, nthreads=4)
    assert res["consensus"] == inst.motif
    assert np.mean(res["sites"] == inst.starts) >= 0.8
