"""Pins of the oracle against the paper's worked example (Figures 1, 2, 4;
Example 1 of Section 5.1) and its hashing examples (Section 6)."""
import itertools

import numpy as np
import pytest

import oracle as O
from tests.conftest import golden_lines

L = 8


def _parse(name):
    out = {}
    for ln in golden_lines(name):
        key, *rest = ln.split()
        out.setdefault(key, []).append(rest)
    return out


@pytest.fixture(scope="module")
def ex(fig1):
    codes = O.encode("".join(fig1).encode())
    seq_off = np.arange(len(fig1) + 1, dtype=np.int64) * 40
    return codes, seq_off


def test_fig1_shape(fig1):
    assert len(fig1) == 7 and all(len(q) == 40 for q in fig1)


def test_fig2_alignment_profile_consensus_score(fig1, ex):
    codes, seq_off = ex
    g = _parse("fig2_alignment.txt")
    starts = [int(v) for v in g["starts"][0]]
    lmers = [r[0] for r in g["lmer"]]
    assert [fig1[i][a - 1:a - 1 + L] for i, a in enumerate(starts)] == lmers
    # the profile P(s) is theta^0 without pseudocount times the bucket size
    lo = O.lmer_offsets(seq_off, L)
    members = np.array([lo[i] + a - 1 for i, a in enumerate(starts)], np.int32)
    prof = np.rint(O.theta0(codes, seq_off, L, members, 0.0) * len(starts)).astype(int)
    row = {"A": 0, "C": 1, "T": 2, "G": 3}
    for r in g["profile"]:
        assert list(prof[:, row[r[0]]]) == [int(v) for v in r[1:]], r[0]
    assert O.consensus(prof.astype(float)) == g["consensus"][0][0]
    sites = np.array(starts, np.int32) - 1
    assert O.score(codes, seq_off, L, sites) == int(g["score"][0][0]) == 53


def test_hash_mapping_examples():
    for word, val in (ln.split() for ln in golden_lines("hash_mapping.txt")):
        codes = O.encode(word.encode())
        off = np.array([0, len(word)], np.int64)
        k = len(word)
        key = O.keys(codes, off, k, np.arange(k, dtype=np.int32))
        assert key.tolist() == [int(val)]


def test_example1_enriched_bucket(fig1, ex):
    codes, seq_off = ex
    g = _parse("fig4_theta0.txt")
    pos = np.array([int(v) - 1 for v in g["positions_read"][0]], np.int32)
    s = int(g["threshold"][0][0])
    keys = O.keys(codes, seq_off, L, pos)
    assert keys.size == 7 * 33
    ck, cc, co, mem = O.enriched(keys, s)
    # "ATGAC" in base 4 with A0 C1 T2 G3, most significant first
    word = g["bucket"][0][0]
    key = 0
    for ch in word:
        key = key * 4 + "ACTG".index(ch)
    assert key == 177
    assert key in ck.tolist()
    c = ck.tolist().index(key)
    assert cc[c] == int(g["bucket_count"][0][0]) == 7
    starts = [int(v) for v in _parse("fig2_alignment.txt")["starts"][0]]
    lo = O.lmer_offsets(seq_off, L)
    assert mem[co[c]:co[c + 1]].tolist() == [lo[i] + a - 1 for i, a in enumerate(starts)]
    # the only other bucket of size >= 4 under this projection
    assert ck.tolist() == [177, 726] and cc.tolist() == [7, 5]
    # bucket sizes over all 231 l-mers
    cnt = O.counts(keys, 5)
    hist = np.bincount(cnt[cnt > 0])
    assert {i: int(v) for i, v in enumerate(hist) if v} == {1: 186, 2: 15, 3: 1, 5: 1, 7: 1}
    assert int(cnt.sum()) == 231


def test_example1_printed_positions_are_garbled(ex):
    """The printed positions do not give bucket ATGAC with the seven l-mers; brute
    force over all 5-subsets shows {1,2,3,6,7} is the only one that does."""
    codes, seq_off = ex
    starts = [int(v) for v in _parse("fig2_alignment.txt")["starts"][0]]
    lo = O.lmer_offsets(seq_off, L)
    target = sorted(lo[i] + a - 1 for i, a in enumerate(starts))
    hits = []
    for P in itertools.combinations(range(L), 5):
        keys = O.keys(codes, seq_off, L, np.array(P, np.int32))
        ck, cc, co, mem = O.enriched(keys, 4)
        for c in range(ck.size):
            if ck[c] == 177 and mem[co[c]:co[c + 1]].tolist() == target:
                hits.append([p + 1 for p in P])
    assert hits == [[1, 2, 3, 6, 7]]


def test_fig4_theta0(ex):
    codes, seq_off = ex
    starts = [int(v) for v in _parse("fig2_alignment.txt")["starts"][0]]
    lo = O.lmer_offsets(seq_off, L)
    members = np.array([lo[i] + a - 1 for i, a in enumerate(starts)], np.int32)
    th = O.theta0(codes, seq_off, L, members, 0.0)
    row = {"A": 0, "C": 1, "T": 2, "G": 3}
    for r in _parse("fig4_theta0.txt")["theta0"]:
        printed = [float(v) for v in r[2:]]  # drop the background column
        assert np.allclose(np.round(th[:, row[r[0]]], 2), printed, atol=0, rtol=0), r[0]
    assert np.allclose(th.sum(axis=1), 1.0)


def test_encode_rejects_non_acgt():
    with pytest.raises(ValueError):
        O.encode(b"ACGTN")
    assert O.encode(b"acgt").tolist() == [0, 1, 3, 2]
