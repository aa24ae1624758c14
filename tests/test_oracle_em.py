"""Pins of the oracle's EM refinement (Section 5.1) and of the Section 5
parameter choice: closed-form special cases, the non-decreasing MAP objective,
probability invariants, brute-force Score optimality on tiny inputs, planted
motif recovery, and the trial bound m against scipy's binomial CDF."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from synth import instance_for_config, planted_instance

IDX = {"A": 0, "C": 1, "T": 2, "G": 3}


def _setup(seqs):
    codes = O.encode("".join(seqs).encode())
    off = np.concatenate([[0], np.cumsum([len(q) for q in seqs])]).astype(np.int64)
    return codes, off


def _random_pwm(rng, l):
    p = rng.random((l, 4)) + 0.05
    return p / p.sum(axis=1, keepdims=True)


def test_one_lmer_per_sequence_closed_form():
    """n_i = l: every posterior is 1, so one M-step gives the column counts of
    all t l-mers with pseudocount, and LL = sum_i log prod_p theta/bg."""
    rng = np.random.default_rng(1)
    l, t, beta = 6, 9, 0.25
    seqs = ["".join("ACGT"[c] for c in rng.integers(0, 4, l)) for _ in range(t)]
    codes, off = _setup(seqs)
    bg = O.background(codes)
    pwm0 = _random_pwm(rng, l)
    # LL of the starting model (0 M-steps)
    _, ll0 = O.em(codes, off, l, bg, pwm0[None], 0, beta)
    want0 = sum(math.log(pwm0[p, IDX[q[p]]] / bg[IDX[q[p]]]) for q in seqs for p in range(l))
    assert ll0[0] == pytest.approx(want0, rel=1e-12, abs=1e-12)
    # one M-step
    pwm1, ll1 = O.em(codes, off, l, bg, pwm0[None], 1, beta)
    cnt = np.zeros((l, 4))
    for q in seqs:
        for p, ch in enumerate(q):
            cnt[p, IDX[ch]] += 1
    want = (cnt + beta) / (t + 4 * beta)
    assert np.allclose(pwm1[0], want, rtol=0, atol=1e-14)
    want1 = sum(math.log(want[p, IDX[q[p]]] / bg[IDX[q[p]]]) for q in seqs for p in range(l))
    assert ll1[0] == pytest.approx(want1, rel=1e-12)


def test_two_lmers_per_sequence_closed_form():
    """n_i = l+1: the posterior of start 0 is the logistic of r0 - r1, and
    LL_i = log((e^r0 + e^r1) / 2)."""
    rng = np.random.default_rng(2)
    l, t, beta = 5, 7, 0.5
    seqs = ["".join("ACGT"[c] for c in rng.integers(0, 4, l + 1)) for _ in range(t)]
    codes, off = _setup(seqs)
    bg = O.background(codes)
    pwm0 = _random_pwm(rng, l)

    def r(q, j):
        return sum(math.log(pwm0[p, IDX[q[j + p]]] / bg[IDX[q[j + p]]]) for p in range(l))

    pwm1, _, lse = O.em(codes, off, l, bg, pwm0[None], 1, beta, want_lse=True)
    cnt = np.zeros((l, 4))
    ll0 = 0.0
    for q in seqs:
        r0, r1 = r(q, 0), r(q, 1)
        z0 = 1.0 / (1.0 + math.exp(r1 - r0))
        ll0 += math.log((math.exp(r0) + math.exp(r1)) / 2.0)
        for p in range(l):
            cnt[p, IDX[q[p]]] += z0
            cnt[p, IDX[q[p + 1]]] += 1.0 - z0
    assert np.allclose(pwm1[0], (cnt + beta) / (t + 4 * beta), rtol=0, atol=1e-13)
    _, ll_start = O.em(codes, off, l, bg, pwm0[None], 0, beta)
    assert ll_start[0] == pytest.approx(ll0, rel=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_map_objective_non_decreasing_and_columns_sum_to_one(seed):
    """Generalised EM with a Dirichlet(1+beta) prior: LL + beta * sum log theta
    never decreases from one E-step to the next."""
    inst = planted_instance(100 + seed, 0, 8, 120, 9, 2)
    codes = O.encode(inst.ascii)
    off = inst.seq_off
    bg = O.background(codes)
    rng = np.random.default_rng(seed)
    beta = 0.25
    pwm = _random_pwm(rng, 9)
    prev = -np.inf
    for it in range(12):
        ll = O.em(codes, off, 9, bg, pwm[None], 0, beta)[1][0]
        obj = ll + beta * np.log(pwm).sum()
        assert obj >= prev - 1e-9 * max(1.0, abs(prev))
        prev = obj
        pwm = O.em(codes, off, 9, bg, pwm[None], 1, beta)[0][0]
        assert np.allclose(pwm.sum(axis=1), 1.0, atol=1e-12)
        assert np.all(pwm > 0)
    # the multi-iteration call gives the same model as chained single steps
    pwm_a, ll_a, tr = O.em(codes, off, 9, bg, _random_pwm(np.random.default_rng(seed), 9)[None],
                           12, beta, want_trace=True)
    assert np.allclose(pwm_a[0], pwm, atol=1e-12)
    assert ll_a[0] == pytest.approx(tr[0, -1])


def test_em_threads_do_not_change_results():
    inst = instance_for_config(1)
    codes = O.encode(inst.ascii)
    rng = np.random.default_rng(3)
    pwm0 = np.stack([_random_pwm(rng, 11) for _ in range(9)])
    bg = O.background(codes)
    a = O.em(codes, inst.seq_off, 11, bg, pwm0, 3, 0.25, nthreads=1)
    b = O.em(codes, inst.seq_off, 11, bg, pwm0, 3, 0.25, nthreads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_sites_are_first_argmax():
    seqs = ["AAAACAAAAC", "CCCCCCCCCC"]
    codes, off = _setup(seqs)
    pwm = np.full((3, 4), 0.1)
    pwm[:, 0] = 0.7  # prefers AAA
    st = O.sites(codes, off, 3, O.background(codes), pwm)
    assert st.tolist() == [0, 0]  # ties -> first start


def test_consensus_tie_goes_to_lowest_code():
    pwm = np.array([[0.25, 0.25, 0.25, 0.25], [0.1, 0.4, 0.1, 0.4], [0.1, 0.1, 0.4, 0.4]])
    assert O.consensus(pwm) == "ACT"


def test_naive_mfp_bound_on_tiny_input():
    """Algorithm 1 (exhaustive search) on a tiny exact-planted instance: the
    pipeline's Score reaches the exhaustive optimum l*t."""
    inst = planted_instance(9, 0, 3, 12, 5, 0)
    seqs = [q.decode() for q in inst.seqs]
    codes, off = _setup(seqs)
    l = 5
    best = 0
    for s in itertools.product(range(12 - l + 1), repeat=3):
        best = max(best, O.score(codes, off, l, np.array(s, np.int32)))
    assert best == l * 3
    res = O.find(seqs, l, 0, k=3, s=3, m=20, seed=1, em_iters=5, beta=0.1)
    assert res["score"] == best


def test_planted_recovery_config1():
    inst = instance_for_config(1)
    res = O.find(inst.seqs, 11, 2, k=7, s=4, m=100, seed=1, em_iters=5, beta=0.25, nthreads=8)
    assert res["consensus"] == inst.motif
    assert np.mean(res["sites"] == inst.starts) >= 0.8


@pytest.mark.parametrize("l,d,k,s,want", [(11, 2, 7, 4, 17), (15, 4, 7, 4, 172),
                                          (18, 6, 8, 3, 2096)])
def test_m_bound_against_scipy(l, d, k, s, want):
    stats = pytest.importorskip("scipy.stats")
    p = math.comb(l - d, k) / math.comb(l, k)
    B = stats.binom.cdf(s - 1, 20, p)
    m = math.ceil(math.log(1 - 0.95) / math.log(B))
    assert O.m_bound(l, d, k, s, 20, 0.95) == m == want


def test_m_bound_undefined_cases():
    assert O.m_bound(11, 2, 10, 4, 20, 0.95) == -1  # k > l-d: p_hat = 0
    assert O.m_bound(11, 2, 7, 4, 20, 1.0) == -1


def test_default_params():
    k, s, m = O.default_params([600] * 20, 15, 4)
    assert k == 10 and s == 3 and m == O.m_bound(15, 4, 10, 3, 20)
    assert O.default_params([600] * 20, 11, 2, k=7, s=4, m=100) == (7, 4, 100)
    # twice the mean bucket size when that exceeds 3
    k, s, m = O.default_params([5000] * 20, 8, 2, k=4)
    assert s == math.ceil(2 * 20 * (5000 - 8 + 1) / 4 ** 4)


# ---------------------------------------------------------------------------
# ZOOPS (zero or one occurrence per sequence, reading R15)
# ---------------------------------------------------------------------------

def _mixture_ll_and_posteriors(seqs, pwm, bg, gamma):
    """Brute force in probability space: for each sequence the mixture
    P(seq) = (1-gamma) prod_b bg(x_b) + sum_j gamma/ns prod_{b not in site} bg(x_b)
    prod_p pwm_p(x_{j+p}), its ratio to the all-background probability, and
    the posterior of each site by Bayes' rule on the joint probabilities."""
    l = pwm.shape[0]
    ll, post = 0.0, []
    for q in seqs:
        x = [IDX[c] for c in q]
        ns = len(q) - l + 1
        p_bg = math.prod(bg[a] for a in x)
        joint_site = []
        for j in range(ns):
            pr = gamma / ns
            for b, a in enumerate(x):
                pr *= pwm[b - j, a] if j <= b < j + l else bg[a]
            joint_site.append(pr)
        total = (1 - gamma) * p_bg + sum(joint_site)
        ll += math.log(total / p_bg)
        post.append([js / total for js in joint_site])
    return ll, post


@pytest.mark.parametrize("gamma", [0.3, 0.8, 1.0])
def test_zoops_matches_mixture_brute_force(gamma):
    """Log-likelihood ratio and one M-step of the ZOOPS oracle against the
    mixture written out in probability space on a tiny input."""
    rng = np.random.default_rng(11)
    l, beta = 4, 0.25
    seqs = ["".join("ACGT"[c] for c in rng.integers(0, 4, n)) for n in (6, 4, 9, 5)]
    codes, off = _setup(seqs)
    bg = O.background(codes)
    pwm0 = _random_pwm(rng, l)
    want_ll, post = _mixture_ll_and_posteriors(seqs, pwm0, bg, gamma)
    _, ll0 = O.em_zoops(codes, off, l, bg, pwm0[None], 0, beta, gamma)
    assert ll0[0] == pytest.approx(want_ll, rel=1e-12, abs=1e-12)
    cnt = np.zeros((l, 4))
    ztot = 0.0
    for q, zq in zip(seqs, post):
        for j, z in enumerate(zq):
            ztot += z
            for p in range(l):
                cnt[p, IDX[q[j + p]]] += z
    pwm1, _ = O.em_zoops(codes, off, l, bg, pwm0[None], 1, beta, gamma)
    assert np.allclose(pwm1[0], (cnt + beta) / (ztot + 4 * beta), rtol=0, atol=1e-13)


def test_zoops_with_gamma_one_is_oops():
    inst = planted_instance(21, 0, 10, 150, 9, 2)
    codes = O.encode(inst.ascii)
    bg = O.background(codes)
    pwm0 = _random_pwm(np.random.default_rng(5), 9)[None]
    a = O.em(codes, inst.seq_off, 9, bg, pwm0, 4, 0.25)
    b = O.em_zoops(codes, inst.seq_off, 9, bg, pwm0, 4, 0.25, 1.0)
    assert np.allclose(a[0], b[0], rtol=0, atol=1e-12)
    assert b[1][0] == pytest.approx(a[1][0], rel=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_zoops_map_objective_non_decreasing(seed):
    """EM on the ZOOPS mixture with a Dirichlet(1+beta) prior: LL + beta *
    sum log theta never decreases; columns sum to one."""
    inst = planted_instance(200 + seed, 0, 12, 140, 9, 2, zoops_frac=0.5)
    codes = O.encode(inst.ascii)
    bg = O.background(codes)
    pwm = _random_pwm(np.random.default_rng(seed), 9)
    prev = -np.inf
    for it in range(10):
        ll = O.em_zoops(codes, inst.seq_off, 9, bg, pwm[None], 0, 0.25, 0.5)[1][0]
        obj = ll + 0.25 * np.log(pwm).sum()
        assert obj >= prev - 1e-9 * max(1.0, abs(prev))
        prev = obj
        pwm = O.em_zoops(codes, inst.seq_off, 9, bg, pwm[None], 1, 0.25, 0.5)[0][0]
        assert np.allclose(pwm.sum(axis=1), 1.0, atol=1e-12)


# --------------------------------------------------------------------------
# Column 0 of theta (Section 5.1, Figure 4): the background model, and the
# ranking rule.  Values are counted by hand from the strings, not recomputed
# by a second implementation.
# --------------------------------------------------------------------------

def test_background_hand_counted_dna():
    """0-order base frequencies in code order A, C, T, G (Section 6's codes);
    a base that never occurs is counted once (reading R7)."""
    # A 2, C 3, T 1, G absent -> 1: total 7
    assert np.array_equal(O.background(O.encode(b"AACCCT")),
                          np.array([2 / 7, 3 / 7, 1 / 7, 1 / 7]))
    # every base present, lower case accepted: A 1, C 1, T 2, G 2 of 6
    assert np.array_equal(O.background(O.encode(b"acgttg")),
                          np.array([1 / 6, 1 / 6, 2 / 6, 2 / 6]))
    # only G: G 5, the three absent bases once each, total 8
    assert np.array_equal(O.background(O.encode(b"GGGGG")),
                          np.array([1 / 8, 1 / 8, 1 / 8, 5 / 8]))
    # the worked example of Figure 1 is near-uniform, as the 0.25 of Figure 4
    # assumes: every base between 0.2 and 0.3
    from conftest import golden_lines
    bg = O.background(O.encode("".join(golden_lines("fig1_sequences.txt")).encode()))
    assert bg.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all((bg > 0.2) & (bg < 0.3))


def test_background_hand_counted_protein():
    """The same rule over the 20 letters ACDEFGHIKLMNPQRSTVWY (codes 0..19)."""
    bg = O.background_a(O.encode_aa(b"WWWY"), 20)
    want = np.full(20, 1 / 22)  # 18 absent letters once each + W 3 + Y 1 = 22
    want[18] = 3 / 22  # W
    want[19] = 1 / 22  # Y
    assert np.array_equal(bg, want)
    bg = O.background_a(O.encode_aa(b"AACD" + b"ACDEFGHIKLMNPQRSTVWY"), 20)
    want = np.full(20, 1 / 24)
    want[0] = 3 / 24  # A: 2 + 1
    want[1] = 2 / 24  # C
    want[2] = 2 / 24  # D
    assert np.array_equal(bg, want)


def test_rank_ties_go_to_the_first_candidate():
    """Ranking (Section 5.1, reading R12): the largest LL wins; among equal LLs
    the candidate earlier in (trial, key) order."""
    assert O.rank(np.array([1.0, 3.0, 3.0, 2.0])) == 1
    assert O.rank(np.array([-5.0, -5.0])) == 0
    assert O.rank(np.array([2.0, 1.0, 7.5, 7.5, 7.5])) == 2
    assert O.rank(np.array([-np.inf, 0.0])) == 1
    assert O.rank(np.array([])) == -1


def test_top_candidates_order():
    """The serving-scale cap keeps the largest buckets; equal sizes keep
    (trial, key) order."""
    cnt = np.array([4, 7, 5, 7, 4, 9])
    assert list(O.top_candidates(cnt, 3)) == [5, 1, 3]
    assert list(O.top_candidates(cnt, 5)) == [5, 1, 3, 2, 0]
    assert list(O.top_candidates(cnt, 10)) == [5, 1, 3, 2, 0, 4]
