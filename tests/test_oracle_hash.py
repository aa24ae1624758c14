"""Pins of the oracle's Philox, projection, hashing and enrichment against
published known-answer vectors, brute-force enumeration and invariants."""
import collections
import math

import numpy as np
import pytest

import oracle as O
from synth import planted_instance
from tests.conftest import golden_lines


def test_philox_known_answers():
    for ln in golden_lines("philox_kat.txt"):
        v = [int(x, 16) for x in ln.split()]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


@pytest.mark.parametrize("l,k", [(8, 5), (11, 7), (15, 7), (18, 8), (20, 10), (32, 16), (5, 5),
                                 (7, 1)])
def test_positions_invariants(l, k):
    seen = set()
    for trial in range(200):
        p = O.positions(12345, trial, l, k)
        assert p.size == k and np.all(np.diff(p) > 0) and p[0] >= 0 and p[-1] < l
        seen.add(tuple(p))
        assert np.array_equal(p, O.positions(12345, trial, l, k))  # deterministic
    if 0 < k < l:
        assert len(seen) > min(100, math.comb(l, k) // 2)


def test_positions_uniform_marginals():
    """Each position is kept with probability k/l (chi-square, 20000 trials)."""
    l, k, T = 11, 7, 20000
    hits = np.zeros(l)
    for trial in range(T):
        hits[O.positions(7, trial, l, k)] += 1
    expect = T * k / l
    var = T * (k / l) * (1 - k / l)
    chi2 = float(((hits - expect) ** 2 / var).sum())
    assert chi2 < 40.0, (hits, chi2)  # df ~ l; 40 is far in the tail


def test_positions_seed_and_trial_change_the_draw():
    a = [tuple(O.positions(1, t, 15, 7)) for t in range(50)]
    b = [tuple(O.positions(2, t, 15, 7)) for t in range(50)]
    assert a != b and len(set(a)) > 30


def test_pack2_bits():
    rng = np.random.default_rng(0)
    codes = rng.integers(0, 4, 1000).astype(np.uint8)
    w = O.pack2(codes)
    assert w.size == (1000 + 15) // 16
    for b in range(1000):
        assert (int(w[b // 16]) >> (2 * (b % 16))) & 3 == codes[b]
    assert int(w[-1]) >> (2 * (1000 % 16)) == 0


def _brute_buckets(seqs, l, pos):
    """All-pairs comparison of projected k-mers (PROJECTION2 of Section 5.2):
    for each l-mer, the ids of all l-mers with an identical projected string."""
    lmers = [q[j:j + l] for q in seqs for j in range(len(q) - l + 1)]
    proj = ["".join(w[p] for p in pos) for w in lmers]
    same = [[h for h in range(len(proj)) if proj[h] == proj[g]] for g in range(len(proj))]
    return lmers, proj, same


@pytest.mark.parametrize("seed", range(6))
def test_enriched_matches_all_pairs_brute_force(seed):
    rng = np.random.default_rng(seed)
    l = int(rng.integers(4, 9))
    k = int(rng.integers(1, l + 1))
    lens = [int(v) for v in rng.integers(l - 1, 30, size=int(rng.integers(1, 6)))]
    lens[0] = max(lens[0], l)
    seqs = ["".join("ACGT"[c] for c in rng.integers(0, 4, n)) for n in lens]
    codes = O.encode("".join(seqs).encode())
    seq_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pos = np.sort(rng.choice(l, k, replace=False)).astype(np.int32)
    keys = O.keys(codes, seq_off, l, pos)
    lmers, proj, same = _brute_buckets(seqs, l, pos)
    assert keys.size == len(lmers)
    # key <-> projected string is one-to-one
    by_key = collections.defaultdict(set)
    for g, kk in enumerate(keys):
        by_key[int(kk)].add(proj[g])
    assert all(len(v) == 1 for v in by_key.values())
    cnt = O.counts(keys, k)
    assert int(cnt.sum()) == len(lmers)
    for g in range(len(lmers)):
        assert cnt[keys[g]] == len(same[g])
    for s in (1, 2, 3, 5):
        ck, cc, co, mem = O.enriched(keys, s)
        got = {tuple(mem[co[c]:co[c + 1]].tolist()) for c in range(ck.size)}
        want = {tuple(v) for v in same if len(v) >= s}
        assert got == want
        assert np.all(np.diff(ck.astype(np.int64)) > 0)
        assert np.all(cc >= s)


def test_ragged_sequences_and_short_ones():
    seqs = ["ACGTACGTAC", "ACG", "ACGTA", "TTTTTTTTTTTTTTTT"]
    lens = [len(q) for q in seqs]
    seq_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    lo = O.lmer_offsets(seq_off, 5)
    assert lo.tolist() == [0, 6, 6, 7, 19]
    codes = O.encode("".join(seqs).encode())
    keys = O.keys(codes, seq_off, 5, np.arange(5, dtype=np.int32))
    assert keys.size == 19
    ck, cc, co, mem = O.enriched(keys, 3)
    # ACGTA (0,1,3,2,0 -> 120) at ids 0, 4 and 6; TTTTT (2 * 341 = 682) twelve
    # times in the last sequence; no l-mer spans two sequences.
    assert ck.tolist() == [120, 682] and cc.tolist() == [3, 12]
    assert mem[co[0]:co[1]].tolist() == [0, 4, 6]
    assert mem[co[1]:co[2]].tolist() == list(range(7, 19))


def test_planted_bucket_appears_in_some_trial():
    inst = planted_instance(5, 0, 20, 600, 11, 2)
    codes = O.encode(inst.ascii)
    h = O.hash_trials(codes, inst.seq_off, 11, 7, 4, 99, 0, 30)
    lo = O.lmer_offsets(inst.seq_off, 11)
    planted = {int(lo[i] + a) for i, a in enumerate(inst.starts)}
    best = 0
    for c in range(h["cand_key"].size):
        mem = set(h["members"][h["cand_off"][c]:h["cand_off"][c + 1]].tolist())
        best = max(best, len(mem & planted))
    assert best >= 4
    # every trial: counts sum to x, cand list sorted by (trial, key)
    order = list(zip(h["cand_trial"].tolist(), h["cand_key"].tolist()))
    assert order == sorted(order) and len(set(order)) == len(order)


def test_top_candidates_order_and_ties():
    cnt = np.array([5, 9, 5, 12, 9, 4, 12, 5])
    assert O.top_candidates(cnt, 5).tolist() == [3, 6, 1, 4, 0]
    assert O.top_candidates(cnt, 100).tolist() == [3, 6, 1, 4, 0, 2, 7, 5]
    # brute force over random lists: same multiset of counts as a full sort,
    # non-increasing counts, ties in index order
    rng = np.random.default_rng(4)
    for _ in range(20):
        c = rng.integers(3, 9, rng.integers(1, 300))
        k = int(rng.integers(1, 320))
        sel = O.top_candidates(c, k)
        assert sel.size == min(k, c.size) and len(set(sel.tolist())) == sel.size
        assert sorted(c[sel].tolist(), reverse=True) == sorted(c.tolist(), reverse=True)[:sel.size]
        for a, b in zip(sel[:-1], sel[1:]):
            assert c[a] > c[b] or (c[a] == c[b] and a < b)
