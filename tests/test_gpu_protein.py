"""The protein-alphabet search (20 letters, keys base 20, FP32 OOPS EM) against
the oracle's find_protein on the same seeded inputs: enriched-bucket totals
and the winner's (trial, key) exactly; the winner's PWM within 1e-5 and its
log-likelihood within 1e-6 relative; consensus, sites and Score identical.
Where the oracle's best two candidates are within the LL tolerance the GPU may
pick either; it is then checked against the oracle's model of its own pick."""
import numpy as np
import pytest

import oracle as O
from synth import planted_protein

from conftest import ll_tol

pytestmark = pytest.mark.gpu


def _run(inst, k, s, m, seed, iters, beta, lower=False):
    import paper_1605_06904_gb300 as P
    ascii = inst.ascii
    if lower:
        ascii = np.frombuffer(bytes(ascii).lower(), np.uint8).copy()
    return P.projection_find_protein(ascii, inst.seq_off, inst.l, k, s, m, seed=seed,
                                     em_iters=iters, pseudocount=beta)


def _check(got, want, inst):
    t, l = inst.t, inst.l
    assert got["n_candidates"] == want["n_candidates"]
    assert got["n_members"] == want["members"].size
    if want["n_candidates"] == 0:
        assert got["win_index"] == -1
        return
    w, g = want["win"], got["win_index"]
    ll = want["ll_all"]
    assert abs(ll[g] - ll[w]) <= ll_tol(ll[w], t), "GPU winner is not a near-tie of the oracle's"
    assert got["win_trial"] == int(want["cand_trial"][g])
    assert got["win_key"] == int(want["cand_key"][g])
    assert np.max(np.abs(got["pwm"] - want["pwm_all"][g])) <= 1e-5
    assert abs(got["loglik"] - ll[g]) <= ll_tol(ll[g], t)
    pwm = want["pwm_all"][g]
    codes = O.encode_aa(bytes(inst.ascii))
    bg = want["bg"]
    sites = O.sites_a(codes, inst.seq_off, l, bg, pwm, 20)
    assert np.array_equal(got["sites"], sites)
    assert got["consensus"] == O.consensus_a(pwm, 20)
    assert got["score"] == O.score_a(codes, inst.seq_off, l, sites, 20)


@pytest.mark.parametrize("case", [
    # (seed, t, n, l, d, k, s, m, iters, beta)
    (7, 15, 200, 10, 2, 4, 3, 30, 5, 0.1),     # l <= 16: 32 candidates per CTA
    (8, 12, 150, 20, 4, 3, 3, 12, 3, 0.25),    # l > 16: 16 candidates per CTA
    (9, 9, 64, 6, 1, 2, 2, 5, 2, 0.5),         # short sequences, many small buckets
    (10, 6, 40, 8, 1, 6, 2, 20, 4, 0.1),       # k = 6, the largest base-20 key
    (15, 30, 600, 12, 3, 4, 3, 10, 3, 0.25),   # x = 17,670 > 16,384: all-pairs enrichment
    (16, 1, 300, 32, 6, 1, 1, 3, 2, 0.25),     # one sequence, l = 32, k = 1, s = 1
])
def test_protein_search_matches_oracle(native_lib, case):
    seed, t, n, l, d, k, s, m, iters, beta = case
    inst = planted_protein(seed, 0, t, n, l, d)
    got = _run(inst, k, s, m, seed, iters, beta)
    want = O.find_protein(inst.seqs, l, k, s, m, seed, iters, beta, nthreads=8)
    _check(got, want, inst)


def test_protein_ragged_and_lower_case(native_lib):
    lens = [33, 120, 17, 250, 64, 91, 12, 200]
    inst = planted_protein(11, 0, len(lens), lens, 12, 2)
    got = _run(inst, 4, 2, 25, 3, 4, 0.25, lower=True)
    want = O.find_protein(inst.seqs, 12, 4, 2, 25, 3, 4, 0.25, nthreads=8)
    _check(got, want, inst)


def test_protein_no_enriched_bucket(native_lib):
    inst = planted_protein(12, 0, 5, 30, 8, 1)
    got = _run(inst, 5, 1000, 3, 0, 2, 0.25)
    assert got["n_candidates"] == 0 and got["win_index"] == -1


def test_protein_rejects_bad_input(native_lib):
    import paper_1605_06904_gb300 as P
    from paper_1605_06904_gb300._native import ProjectionError
    inst = planted_protein(13, 0, 4, 40, 8, 1)
    bad = inst.ascii.copy()
    bad[57] = ord("B")
    with pytest.raises(ProjectionError) as e:
        P.projection_find_protein(bad, inst.seq_off, 8, 3, 2, 4)
    assert e.value.status == -6 and "57" in str(e.value)
    with pytest.raises(ProjectionError) as e:
        P.projection_find_protein(inst.ascii, inst.seq_off, 8, 7, 2, 4)
    assert e.value.status == -1


def test_protein_search_is_deterministic(native_lib):
    inst = planted_protein(14, 0, 24, 300, 12, 3)
    a = _run(inst, 4, 3, 20, 5, 5, 0.25)
    b = _run(inst, 4, 3, 20, 5, 5, 0.25)
    assert a["win_index"] == b["win_index"] and a["loglik"] == b["loglik"]
    assert np.array_equal(a["pwm"], b["pwm"]) and np.array_equal(a["sites"], b["sites"])
