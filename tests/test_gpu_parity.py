"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer work (packing, projection positions, keys, bucket counts, enriched
lists) must match bit for bit.  Floating point: theta^0 within 1e-6, EM PWM
entries within 1e-5 absolute and per-candidate log-likelihood ratios within
1e-6 relative (scale floored at t nats) for the FP32 path; consensus and sites
identical."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import instance_for_config, planted_instance
from tests.conftest import ll_tol, oracle_theta0_sample

pytestmark = pytest.mark.gpu

PWM_TOL = 1e-5


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


def upload(P, ascii_bytes):
    a = torch.from_numpy(np.frombuffer(bytes(ascii_bytes), np.uint8).copy()).cuda()
    return P.projection_pack(a)


def inst_arrays(inst):
    codes = O.encode(inst.ascii)
    return codes, inst.seq_off


def hash_np(h):
    return {
        "cand_trial": h["cand_trial"].cpu().numpy(),
        "cand_key": h["cand_key"].cpu().numpy().view(np.uint32),
        "cand_cnt": h["cand_cnt"].cpu().numpy(),
        "cand_off": h["cand_off"].cpu().numpy(),
        "members": h["members"].cpu().numpy(),
    }


def assert_hash_equal(got, want):
    for key in ("cand_trial", "cand_key", "cand_cnt", "cand_off", "members"):
        g, w = np.asarray(got[key]), np.asarray(want[key])
        assert g.shape == w.shape, (key, g.shape, w.shape)
        assert np.array_equal(g.astype(np.int64), w.astype(np.int64)), key


# ---------------------------------------------------------------------------
# a1 pack, background
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 15, 16, 17, 33, 1000, 100003])
def test_pack_bit_exact(P, n):
    rng = np.random.default_rng(n)
    ascii_ = np.frombuffer(b"ACGTacgt", np.uint8)[rng.integers(0, 8, n)].tobytes()
    got = upload(P, ascii_).cpu().numpy().view(np.uint32)
    want = O.pack2(O.encode(ascii_))
    assert np.array_equal(got[:want.size], want)


def test_pack_rejects_non_acgt(P):
    a = bytearray(b"ACGT" * 100)
    a[123] = ord("N")
    a[301] = ord("-")
    with pytest.raises(P.ProjectionError) as e:
        upload(P, bytes(a))
    assert e.value.status == -6 and "123" in str(e.value)


@pytest.mark.parametrize("cfg", [1, 5])
def test_background_matches_oracle(P, cfg):
    inst = instance_for_config(cfg) if cfg == 1 else planted_instance(3, 0, 50, 500, 20, 5,
                                                                      background="markov_gc40")
    packed = upload(P, inst.ascii)
    bg = P.projection_background(packed, inst.seq_off[-1]).cpu().numpy()
    assert np.array_equal(bg, O.background(O.encode(inst.ascii)))


def test_background_missing_base_counts_once(P):
    packed = upload(P, b"AAAACCCC")
    bg = P.projection_background(packed, 8).cpu().numpy()
    assert np.array_equal(bg, O.background(O.encode(b"AAAACCCC")))


# ---------------------------------------------------------------------------
# a2 positions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("l,k", [(8, 5), (11, 7), (15, 7), (18, 8), (20, 10), (32, 10), (9, 9),
                                 (12, 1)])
@pytest.mark.parametrize("seed", [0, 1001, 2**63 + 12345])
def test_positions_bit_exact(P, l, k, seed):
    T0, T = 5, 300
    got = P.projection_positions(seed, T0, T, l, k).cpu().numpy()
    want = np.stack([O.positions(seed, T0 + i, l, k) for i in range(T)])
    assert np.array_equal(got, want)


# ---------------------------------------------------------------------------
# a3-a5 project, hash, count, enrich
# ---------------------------------------------------------------------------

def test_worked_example_bucket(P, fig1):
    ascii_ = "".join(fig1).encode()
    packed = upload(P, ascii_)
    off = np.arange(8, dtype=np.int64) * 40
    pos = np.array([0, 1, 2, 5, 6], np.int32)  # Example 1, 1-based {1,2,3,6,7}
    h = P.trial_hash(packed, off, 8, 5, 4, 0, 0, 1, positions_in=pos, want_counts=True)
    g = hash_np(h)
    assert g["cand_key"].tolist() == [177, 726] and g["cand_cnt"].tolist() == [7, 5]
    lo = O.lmer_offsets(off, 8)
    starts = (8, 19, 3, 5, 31, 27, 15)
    assert g["members"][:7].tolist() == [lo[i] + a - 1 for i, a in enumerate(starts)]
    codes = O.encode(ascii_)
    want = O.hash_trials(codes, off, 8, 5, 4, 0, 0, 1, pos_override=pos, with_counts=True)
    assert_hash_equal(g, want)
    assert np.array_equal(h["counts"].cpu().numpy().view(np.uint32), want["counts"])


@pytest.mark.parametrize("nt", [1024, 512])
@pytest.mark.parametrize("cfg,trials", [(1, (0, 100)), (2, (0, 172)), (3, (0, 150)),
                                        (3, (1850, 150)), (5, (0, 3)), (5, (497, 3))])
def test_hash_configs_bit_exact(P, cfg, trials, nt, monkeypatch):
    """Both CTA sizes of the bucket kernels (the hash-tile autotuner's choices;
    the serving-scale input keeps 1024, its units need a whole SM)."""
    monkeypatch.setenv("PROJ_HASH_NT", str(nt))
    inst = instance_for_config(cfg)
    prm = inst.params
    codes, off = inst_arrays(inst)
    packed = upload(P, inst.ascii)
    t0, T = trials
    h = P.trial_hash(packed, off, inst.l, prm["k"], prm["s"], 1000 + cfg, t0, T,
                     want_positions=True, want_counts=(T <= 100))
    want = O.hash_trials(codes, off, inst.l, prm["k"], prm["s"], 1000 + cfg, t0, t0 + T,
                         with_counts=(T <= 100))
    assert_hash_equal(hash_np(h), want)
    assert np.array_equal(h["positions"].cpu().numpy(), want["positions"])
    if T <= 100:
        cnt = h["counts"].cpu().numpy().view(np.uint32)
        assert np.array_equal(cnt, want["counts"])
        assert np.all(cnt.sum(axis=1) == inst.n_lmers)  # every l-mer lands in one bucket


def _random_case(seed, t, nmin, nmax, alphabet=b"ACGT"):
    rng = np.random.default_rng(seed)
    lens = rng.integers(nmin, nmax + 1, t)
    seqs = [np.frombuffer(alphabet, np.uint8)[rng.integers(0, len(alphabet), n)].tobytes()
            for n in lens]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return b"".join(seqs), off


@pytest.mark.parametrize("case", [
    dict(seed=1, t=7, nmin=8, nmax=60, l=8, k=5, s=1),       # every l-mer enriched
    dict(seed=2, t=7, nmin=8, nmax=60, l=8, k=8, s=2),       # k = l
    dict(seed=3, t=5, nmin=9, nmax=9, l=9, k=3, s=2),        # one l-mer per sequence
    dict(seed=4, t=1, nmin=500, nmax=500, l=12, k=4, s=5),   # a single sequence
    dict(seed=5, t=9, nmin=11, nmax=300, l=11, k=1, s=50),   # k = 1
    dict(seed=6, t=20, nmin=590, nmax=610, l=15, k=7, s=10**6),  # nothing enriched
    dict(seed=7, t=30, nmin=200, nmax=2500, l=14, k=8, s=3),  # u16 histogram
    dict(seed=8, t=6, nmin=19000, nmax=21000, l=16, k=9, s=2),  # u32, 8 key-range parts
    dict(seed=9, t=40, nmin=400, nmax=600, l=20, k=10, s=2),  # u16, 16 parts
    dict(seed=10, t=4, nmin=100000, nmax=100000, l=12, k=8, s=4),  # input not staged in smem
    dict(seed=11, t=12, nmin=40, nmax=200, l=32, k=10, s=2),  # l = 32
    # partitioned mode over many short sequences: staged and unstaged chunks
    dict(seed=12, t=12000, nmin=24, nmax=30, l=20, k=10, s=2),
    dict(seed=13, t=30000, nmin=21, nmax=22, l=20, k=10, s=2),
])
@pytest.mark.parametrize("nt", [1024, 512])
def test_hash_edge_cases_bit_exact(P, case, nt, monkeypatch):
    monkeypatch.setenv("PROJ_HASH_NT", str(nt))
    ascii_, off = _random_case(case["seed"], case["t"], case["nmin"], case["nmax"])
    l, k, s = case["l"], case["k"], case["s"]
    codes = O.encode(ascii_)
    packed = upload(P, ascii_)
    T = 3
    h = P.trial_hash(packed, off, l, k, s, case["seed"], 0, T, want_counts=(k <= 9))
    want = O.hash_trials(codes, off, l, k, s, case["seed"], 0, T, with_counts=(k <= 9))
    assert_hash_equal(hash_np(h), want)
    if k <= 9:
        assert np.array_equal(h["counts"].cpu().numpy().view(np.uint32), want["counts"])


def test_hash_degenerate_single_base_input(P):
    ascii_ = b"A" * 3000 + b"C" * 70
    off = np.array([0, 1500, 3000, 3070], np.int64)
    codes = O.encode(ascii_)
    packed = upload(P, ascii_)
    h = P.trial_hash(packed, off, 10, 6, 3, 5, 0, 2)
    want = O.hash_trials(codes, off, 10, 6, 3, 5, 0, 2)
    assert_hash_equal(hash_np(h), want)
    assert int(want["cand_cnt"].max()) == 2 * (1500 - 10 + 1)


def test_hash_partitioned_unit_beyond_u16(P):
    """A key-range part of one trial holding more than 65,535 l-mers (a long run
    of one base puts them all in bucket 0): the counting pass counts that unit in
    two rounds of u32 counters instead of u16 ones; lists and counts stay
    bit-exact (Algorithm 2 steps 2c-3)."""
    rng = np.random.default_rng(14)
    tail = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 3000)].tobytes()
    ascii_ = b"A" * 90000 + tail
    off = np.array([0, 90000, 93000], np.int64)
    codes = O.encode(ascii_)
    packed = upload(P, ascii_)
    h = P.trial_hash(packed, off, 16, 9, 2, 14, 0, 2, want_counts=True)
    want = O.hash_trials(codes, off, 16, 9, 2, 14, 0, 2, with_counts=True)
    assert_hash_equal(hash_np(h), want)
    assert np.array_equal(h["counts"].cpu().numpy().view(np.uint32), want["counts"])
    assert int(want["cand_cnt"].max()) == 90000 - 16 + 1


def test_hash_capacity_overflow_reports_totals(P, native_lib):
    inst = instance_for_config(1)
    packed = upload(P, inst.ascii)
    off = np.ascontiguousarray(inst.seq_off)
    import ctypes
    dev = packed.device
    cap_c, cap_m = 5, 7
    bufs = [torch.zeros(cap_c, dtype=torch.int32, device=dev) for _ in range(3)]
    co = torch.zeros(cap_c + 1, dtype=torch.int64, device=dev)
    mem = torch.full((cap_m,), -7, dtype=torch.int32, device=dev)
    tot = torch.zeros(2, dtype=torch.int64, device=dev)
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())
    rc = native_lib.trial_hash(ptr(packed), ctypes.c_void_p(off.ctypes.data), inst.t, 11, 7, 4,
                               1001, 0, 10, None, None, None, cap_c, cap_m, ptr(bufs[0]),
                               ptr(bufs[1]), ptr(bufs[2]), ptr(co), ptr(mem), ptr(tot),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    C, M = tot.cpu().tolist()
    want = O.hash_trials(O.encode(inst.ascii), inst.seq_off, 11, 7, 4, 1001, 0, 10)
    assert C == want["cand_key"].size and M == want["members"].size
    assert C > cap_c and M > cap_m
    # the candidates that fit are the first ones of the full list
    assert np.array_equal(bufs[1].cpu().numpy().view(np.uint32), want["cand_key"][:cap_c])


# ---------------------------------------------------------------------------
# a6 theta^0, a7-a8 EM, a9 finalize
# ---------------------------------------------------------------------------

def _candidates(P, inst, cfg_seed, trials=None):
    prm = inst.params
    packed = upload(P, inst.ascii)
    m = trials if trials is not None else prm["m"] or O.default_params(
        inst.lens, inst.l, inst.d, prm["k"], prm["s"], 0)[2]
    h = P.trial_hash(packed, inst.seq_off, inst.l, prm["k"], prm["s"], cfg_seed, 0, m)
    return packed, h


@pytest.mark.parametrize("cfg", [1, 2])
def test_theta0_matches_oracle(P, cfg):
    inst = instance_for_config(cfg)
    codes = O.encode(inst.ascii)
    prm = inst.params
    oh = O.hash_trials(codes, inst.seq_off, inst.l, prm["k"], prm["s"], 1000 + cfg, 0, 40)
    want = O.theta0_all(codes, inst.seq_off, inst.l, oh["cand_off"], oh["members"], 0.25)
    packed = upload(P, inst.ascii)
    co = torch.from_numpy(oh["cand_off"].astype(np.int64)).cuda()
    mem = torch.from_numpy(oh["members"].astype(np.int32)).cuda()
    th = P.theta0_build(packed, inst.seq_off, inst.l, co, mem, oh["cand_key"].size, 0.25)
    assert np.max(np.abs(th.cpu().numpy() - want)) <= 1e-6


@pytest.mark.parametrize("form", ["warp", "thread"])
def test_theta0_large_and_many_buckets(P, form):
    """theta0 (Example 1, Figure 4) in both kernel forms: a few large buckets
    (one warp per candidate; a bucket of every l-mer passes the 255-per-lane
    fold of the 8-bit counters, plus an empty and a one-member bucket) and more
    than 65,536 small ones (one thread per candidate)."""
    inst = instance_for_config(2)
    codes = O.encode(inst.ascii)
    x = int((inst.lens - inst.l + 1).sum())
    rng = np.random.default_rng(5)
    if form == "warp":
        lists = [np.arange(x), np.zeros(0, np.int64), np.array([5]),
                 np.sort(rng.choice(x, 300, replace=False))]
    else:
        lists = [np.sort(rng.choice(x, int(rng.integers(1, 5)), replace=False))
                 for _ in range(70_000)]
    cand_off = np.zeros(len(lists) + 1, np.int64)
    cand_off[1:] = np.cumsum([len(a) for a in lists])
    members = np.concatenate(lists).astype(np.int32)
    want = O.theta0_all(codes, inst.seq_off, inst.l, cand_off, members, 0.25)
    packed = upload(P, inst.ascii)
    co = torch.from_numpy(cand_off).cuda()
    mem = torch.from_numpy(members).cuda()
    th = P.theta0_build(packed, inst.seq_off, inst.l, co, mem, len(lists), 0.25)
    assert np.max(np.abs(th.cpu().numpy() - want)) <= 1e-6


def _em_case(P, inst, theta0_f32, iters, beta, precision):
    codes = O.encode(inst.ascii)
    packed = upload(P, inst.ascii)
    bg = P.projection_background(packed, inst.seq_off[-1])
    th0 = torch.from_numpy(theta0_f32).cuda()
    th, ll = P.em_refine(packed, inst.seq_off, inst.l, bg, th0, iters, beta, precision)
    w_pwm, w_ll = O.em(codes, inst.seq_off, inst.l, O.background(codes),
                       theta0_f32.astype(np.float64), iters, beta, nthreads=8)
    return th.cpu().numpy(), ll.cpu().numpy(), w_pwm, w_ll


def _sample_theta0(P, inst, seed, n, trials=30):
    return oracle_theta0_sample(inst, inst.params["k"], inst.params["s"], seed, n, trials)


@pytest.mark.parametrize("cfg,n,iters", [(1, 300, 5), (1, 9, 5), (2, 200, 5), (3, 64, 8),
                                         (1, 40, 0)])
def test_em_fp32_matches_oracle(P, cfg, n, iters):
    inst = instance_for_config(cfg)
    th0 = _sample_theta0(P, inst, 1000 + cfg, n)
    pwm, ll, w_pwm, w_ll = _em_case(P, inst, th0, iters, 0.25, P.PROJ_EM_FP32)
    assert np.max(np.abs(pwm - w_pwm)) <= PWM_TOL
    assert np.all(np.abs(ll - w_ll) <= ll_tol(w_ll, inst.t))
    assert np.allclose(pwm.sum(axis=2), 1.0, atol=1e-5)


def test_em_fp32_ragged_sequences(P):
    inst = planted_instance(77, 0, 13, [60, 500, 33, 900, 250, 17, 1200, 64, 400, 19, 700, 88,
                                        301], 15, 3)
    rng = np.random.default_rng(5)
    th0 = rng.random((37, 15, 4)).astype(np.float32) + 0.05
    th0 = (th0 / th0.sum(axis=2, keepdims=True)).astype(np.float32)
    pwm, ll, w_pwm, w_ll = _em_case(P, inst, th0, 5, 0.25, P.PROJ_EM_FP32)
    assert np.max(np.abs(pwm - w_pwm)) <= PWM_TOL
    assert np.all(np.abs(ll - w_ll) <= ll_tol(w_ll, inst.t))


def test_em_fp32_is_deterministic(P):
    inst = instance_for_config(1)
    th0 = _sample_theta0(P, inst, 1001, 50)
    packed = upload(P, inst.ascii)
    bg = P.projection_background(packed, inst.seq_off[-1])
    t0 = torch.from_numpy(th0).cuda()
    a = P.em_refine(packed, inst.seq_off, inst.l, bg, t0, 5, 0.25)
    b = P.em_refine(packed, inst.seq_off, inst.l, bg, t0, 5, 0.25)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def _check_find(got, want, inst, codes):
    assert got["n_candidates"] == want["n_candidates"]
    assert got["k"] == want["k"] and got["s"] == want["s"] and got["m"] == want["m"]
    assert got["consensus"] == want["consensus"]
    assert abs(got["loglik"] - want["loglik"]) <= ll_tol(want["loglik"], inst.t)
    if got["win_index"] != want["win"]:
        # a different candidate of (numerically) equal likelihood: allowed
        assert abs(want["ll_all"][got["win_index"]] - want["loglik"]) <= ll_tol(
            want["loglik"], inst.t)
    assert np.max(np.abs(got["pwm"] - want["pwm"])) <= PWM_TOL
    if not np.array_equal(got["sites"], want["sites"]):
        # only a tie within FP32 noise may move a site
        W = np.log(want["pwm"]) - np.log(want["bg"])[None, :]
        for i in np.nonzero(got["sites"] != want["sites"])[0]:
            q = codes[inst.seq_off[i]:inst.seq_off[i + 1]]
            r = lambda j: sum(W[p, q[j + p]] for p in range(inst.l))
            assert abs(r(got["sites"][i]) - r(want["sites"][i])) <= 1e-4
    assert got["score"] == O.score(codes, inst.seq_off, inst.l, got["sites"])


def test_find_config1_matches_oracle(P):
    inst = instance_for_config(1)
    prm = inst.params
    got = P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, prm["k"], prm["s"],
                            prm["m"], seed=1001, em_iters=prm["em_iters"],
                            pseudocount=prm["beta"])
    want = O.find([q.decode() for q in inst.seqs], inst.l, inst.d, prm["k"], prm["s"], prm["m"],
                  seed=1001, em_iters=prm["em_iters"], beta=prm["beta"], nthreads=8)
    codes = O.encode(inst.ascii)
    _check_find(got, want, inst, codes)
    assert got["consensus"] == inst.motif  # planted motif recovered


def test_find_packed_equals_find(P):
    inst = instance_for_config(1)
    prm = inst.params
    a = P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, prm["k"], prm["s"], 30,
                          seed=5, em_iters=3)
    packed = upload(P, inst.ascii)
    b = P.projection_find_packed(packed, inst.seq_off, inst.l, inst.d, prm["k"], prm["s"], 30,
                                 seed=5, em_iters=3)
    for key in ("n_candidates", "win_index", "win_trial", "win_key", "loglik", "score",
                "consensus"):
        assert a[key] == b[key], key
    assert np.array_equal(a["pwm"], b["pwm"]) and np.array_equal(a["sites"], b["sites"])


def test_find_rejects_bad_input(P):
    with pytest.raises(P.ProjectionError) as e:
        P.projection_find(np.frombuffer(b"ACGTNACGTACGT", np.uint8), [0, 13], 5, 1, 3, 2, 4)
    assert e.value.status == -6
    with pytest.raises(P.ProjectionError) as e:
        P.projection_find(np.frombuffer(b"ACGTACGT", np.uint8), [0, 4, 8], 5, 1, 3, 2, 4)
    assert e.value.status == -1  # a sequence shorter than l


def test_find_config2_full_size(P):
    """Config 2 at full size: the whole path (projection_find) against the
    oracle's whole path, plus the step-wise ABI (the kernels the whole path
    launches, in the same configuration) with every trial's buckets bit-exact
    and EM on a sample of candidates."""
    inst = instance_for_config(2)
    prm = inst.params
    k, s, m = O.default_params(inst.lens, inst.l, inst.d, prm["k"], prm["s"], 0)
    assert m == 172
    codes, off = inst_arrays(inst)
    got = P.projection_find(inst.ascii, off, inst.l, inst.d, prm["k"], prm["s"], 0, seed=1002,
                            em_iters=5, pseudocount=0.25)
    want = O.find([q.decode() for q in inst.seqs], inst.l, inst.d, prm["k"], prm["s"], 0,
                  seed=1002, em_iters=5, beta=0.25, nthreads=16, with_hash=True)
    _check_find(got, want, inst, codes)
    packed = upload(P, inst.ascii)
    h = P.trial_hash(packed, off, inst.l, k, s, 1002, 0, m)
    assert_hash_equal(hash_np(h), want["hash"])
    C = h["n_candidates"]
    th0 = P.theta0_build(packed, off, inst.l, h["cand_off"], h["members"], C, 0.25)
    bg = P.projection_background(packed, off[-1])
    th, ll = P.em_refine(packed, off, inst.l, bg, th0, 5, 0.25)
    fin = P.projection_finalize(packed, off, inst.l, bg, th, ll)
    sample = np.unique(np.concatenate([np.arange(0, C, 97), [fin["best"]]]))
    assert np.max(np.abs(th.cpu().numpy()[sample] - want["pwm_all"][sample])) <= PWM_TOL
    assert np.all(np.abs(ll.cpu().numpy()[sample] - want["ll_all"][sample]) <=
                  ll_tol(want["ll_all"][sample], inst.t))
    assert fin["consensus"] == want["consensus"]


@pytest.mark.parametrize("precision", ["fp32", "bf16split"])
def test_em_refine_sites_of_every_candidate(P, precision):
    """em_refine's sites_out: per candidate, Definition 1's start vector under
    its final model (first start of highest r, FP64), identical to the oracle's
    `sites` evaluated on the same model, for 300 candidates of config 1."""
    inst = instance_for_config(1)
    th0 = _sample_theta0(P, inst, 1001, 300)
    codes = O.encode(inst.ascii)
    packed = upload(P, inst.ascii)
    bg = P.projection_background(packed, inst.seq_off[-1])
    prec = P.PROJ_EM_FP32 if precision == "fp32" else P.PROJ_EM_BF16_SPLIT
    th, ll, st = P.em_refine(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(), 5,
                             0.25, prec, want_sites=True)
    th, st = th.cpu().numpy().astype(np.float64), st.cpu().numpy()
    assert st.shape == (th0.shape[0], inst.t)
    obg = O.background(codes)
    for c in range(th.shape[0]):
        assert np.array_equal(st[c], O.sites(codes, inst.seq_off, inst.l, obg, th[c])), c
    # the models themselves still match the oracle's
    w_pwm, _ = O.em(codes, inst.seq_off, inst.l, obg, th0.astype(np.float64), 5, 0.25, nthreads=8)
    assert np.max(np.abs(th - w_pwm)) <= (PWM_TOL if precision == "fp32" else 5e-5)


def test_em_refine_zoops_sites_of_every_candidate(P):
    """The same output of the ZOOPS refinement (sites as for OOPS: the first
    start of highest score in every sequence)."""
    inst = instance_for_config(1)
    th0 = _sample_theta0(P, inst, 1001, 64)
    codes = O.encode(inst.ascii)
    packed = upload(P, inst.ascii)
    bg = P.projection_background(packed, inst.seq_off[-1])
    th, ll, st = P.em_refine_zoops(packed, inst.seq_off, inst.l, bg, torch.from_numpy(th0).cuda(),
                                   5, 0.25, 0.6, P.PROJ_EM_FP32, want_sites=True)
    th, st = th.cpu().numpy().astype(np.float64), st.cpu().numpy()
    obg = O.background(codes)
    for c in range(th.shape[0]):
        assert np.array_equal(st[c], O.sites(codes, inst.seq_off, inst.l, obg, th[c])), c


@pytest.mark.parametrize("nt", ["1024", "512"])
def test_find_with_each_hash_cta_size(P, nt, monkeypatch):
    """A whole search with each bucket-kernel CTA size gives the same result."""
    monkeypatch.setenv("PROJ_HASH_NT", nt)
    inst = instance_for_config(1)
    prm = inst.params
    r = P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, prm["k"], prm["s"], 30,
                          seed=5, em_iters=3, pseudocount=0.25)
    monkeypatch.setenv("PROJ_HASH_NT", "1024")
    q = P.projection_find(inst.ascii, inst.seq_off, inst.l, inst.d, prm["k"], prm["s"], 30,
                          seed=5, em_iters=3, pseudocount=0.25)
    for key in ("n_candidates", "n_members", "win_index", "consensus", "loglik", "score"):
        assert r[key] == q[key], key
