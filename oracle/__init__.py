"""FP64 CPU oracle of the PROJECTION motif finder -- TEST INFRASTRUCTURE ONLY.

Thin numpy wrapper around ``projection_oracle.c`` (plain C, IEEE double).  It
states, step by step, what Clemente, Cabarle & Adorna (arXiv 1605.06904)
describe: Algorithm 2 (project, hash, enriched buckets), the Section 5
parameter choice, and the EM refinement of Section 5.1 (OOPS model).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It imports nothing from the CUDA library
and the CUDA library imports nothing from it.

Every function is pinned by a CPU test (see ``tests/test_oracle_*.py``); none is
"parity unpinned" except where its docstring says so.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "projection_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_projection_oracle.so")
_lock = threading.Lock()
_lib = None

LETTERS = "ACTG"  # code order of Section 6: A:0, C:1, T:2, G:3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-D_GNU_SOURCE",
           _SRC, "-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            lib.orc_encode.argtypes = [P, i64, P]; lib.orc_encode.restype = i64
            lib.orc_pack2.argtypes = [P, i64, P]; lib.orc_pack2.restype = None
            lib.orc_philox4x32_10.argtypes = [P, P, P]; lib.orc_philox4x32_10.restype = None
            lib.orc_positions.argtypes = [u64, u64, i32, i32, P]; lib.orc_positions.restype = i32
            lib.orc_lmer_offsets.argtypes = [P, i32, i32, P]; lib.orc_lmer_offsets.restype = i64
            lib.orc_keys.argtypes = [P, P, i32, i32, i32, P, P]; lib.orc_keys.restype = None
            lib.orc_counts.argtypes = [P, i64, i32, P]; lib.orc_counts.restype = None
            lib.orc_enriched.argtypes = [P, i64, i32, P, P, P, P, i64, i64, P]
            lib.orc_enriched.restype = i64
            lib.orc_m_bound.argtypes = [i32, i32, i32, i32, i32, f64]; lib.orc_m_bound.restype = i64
            lib.orc_background.argtypes = [P, i64, P]; lib.orc_background.restype = None
            lib.orc_theta0.argtypes = [P, P, P, i32, i32, P, i32, f64, P]
            lib.orc_theta0.restype = None
            lib.orc_em.argtypes = [P, P, i32, i32, P, P, i64, i32, f64, P, P, P, i32]
            lib.orc_em.restype = i32
            lib.orc_em_zoops.argtypes = [P, P, i32, i32, P, P, i64, i32, f64, f64, P, P, i32]
            lib.orc_em_zoops.restype = i32
            lib.orc_encode_aa.argtypes = [P, i64, P]
            lib.orc_encode_aa.restype = i64
            lib.orc_keys_a.argtypes = [P, P, i32, i32, i32, P, i32, P]
            lib.orc_keys_a.restype = None
            lib.orc_background_a.argtypes = [P, i64, i32, P]
            lib.orc_background_a.restype = None
            lib.orc_theta0_a.argtypes = [P, P, P, i32, i32, P, i32, f64, i32, P]
            lib.orc_theta0_a.restype = None
            lib.orc_em_a.argtypes = [P, P, i32, i32, i32, P, P, i64, i32, f64, P, i32]
            lib.orc_em_a.restype = i32
            lib.orc_sites_a.argtypes = [P, P, i32, i32, i32, P, P, P]
            lib.orc_sites_a.restype = None
            lib.orc_consensus_a.argtypes = [P, i32, i32, ctypes.c_char_p, ctypes.c_char_p]
            lib.orc_consensus_a.restype = None
            lib.orc_score_a.argtypes = [P, P, i32, i32, i32, P]
            lib.orc_score_a.restype = i32
            lib.orc_sites.argtypes = [P, P, i32, i32, P, P, P]; lib.orc_sites.restype = None
            lib.orc_consensus.argtypes = [P, i32, P]; lib.orc_consensus.restype = None
            lib.orc_score.argtypes = [P, P, i32, i32, P]; lib.orc_score.restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Alphabet, packing, Philox, positions (Section 6; Algorithm 2 step 2a)
# --------------------------------------------------------------------------

def encode(ascii_bytes) -> np.ndarray:
    """ASCII A/C/G/T (any case) -> codes A0 C1 T2 G3.  Raises ValueError naming
    the first other character."""
    a = np.frombuffer(bytes(ascii_bytes), dtype=np.uint8) if not isinstance(
        ascii_bytes, np.ndarray) else _c(ascii_bytes, np.uint8)
    out = np.empty(a.size, np.uint8)
    bad = _L().orc_encode(_p(a), a.size, _p(out))
    if bad >= 0:
        raise ValueError(f"character {chr(a[bad])!r} at index {bad} is not A/C/G/T")
    return out


def pack2(codes: np.ndarray) -> np.ndarray:
    codes = _c(codes, np.uint8)
    out = np.empty((codes.size + 15) // 16, np.uint32)
    _L().orc_pack2(_p(codes), codes.size, _p(out))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32); k = _c(key, np.uint32); o = np.empty(4, np.uint32)
    _L().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def positions(seed: int, trial: int, l: int, k: int) -> np.ndarray:
    out = np.empty(k, np.int32)
    if _L().orc_positions(seed & (2**64 - 1), trial, l, k, _p(out)) != 0:
        raise ValueError("need 1 <= k <= l <= 32")
    return out


# --------------------------------------------------------------------------
# l-mers, keys, buckets, enrichment (Algorithm 2 steps 2b, 2c, 3)
# --------------------------------------------------------------------------

def lmer_offsets(seq_off: np.ndarray, l: int) -> np.ndarray:
    seq_off = _c(seq_off, np.int64)
    t = seq_off.size - 1
    out = np.empty(t + 1, np.int64)
    _L().orc_lmer_offsets(_p(seq_off), t, l, _p(out))
    return out


def keys(codes, seq_off, l, pos) -> np.ndarray:
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64); pos = _c(pos, np.int32)
    t = seq_off.size - 1
    x = int(lmer_offsets(seq_off, l)[-1])
    out = np.empty(x, np.uint32)
    _L().orc_keys(_p(codes), _p(seq_off), t, l, pos.size, _p(pos), _p(out))
    return out


def counts(keys_: np.ndarray, k: int) -> np.ndarray:
    keys_ = _c(keys_, np.uint32)
    out = np.empty(4 ** k, np.uint32)
    _L().orc_counts(_p(keys_), keys_.size, k, _p(out))
    return out


def enriched(keys_: np.ndarray, s: int):
    """Buckets with >= s l-mers for one trial: (cand_key, cand_cnt, cand_off[C+1], members)."""
    keys_ = _c(keys_, np.uint32)
    x = keys_.size
    cap_c = max(1, x // max(s, 1) + 1)
    ck = np.empty(cap_c, np.uint32); cc = np.empty(cap_c, np.int32)
    co = np.empty(cap_c + 1, np.int64); mem = np.empty(max(x, 1), np.int32)
    nm = np.zeros(1, np.int64)
    nc = _L().orc_enriched(_p(keys_), x, s, _p(ck), _p(cc), _p(co), _p(mem), cap_c, max(x, 1),
                           _p(nm))
    nc = int(nc); nmv = int(nm[0])
    co[nc] = nmv
    return ck[:nc].copy(), cc[:nc].copy(), co[:nc + 1].copy(), mem[:nmv].copy()


def hash_trials(codes, seq_off, l, k, s, seed, trial_begin, trial_end, pos_override=None,
                with_counts=False):
    """Algorithm 2 steps 2-3 for trials [trial_begin, trial_end): CSR candidate
    list sorted by (trial, key); members ascending global l-mer ids."""
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64)
    T = trial_end - trial_begin
    pos_all = np.empty((T, k), np.int32)
    ct, ck, cc, offs, mems, cnts = [], [], [], [], [], []
    base = 0
    for ti in range(T):
        trial = trial_begin + ti
        pos = positions(seed, trial, l, k) if pos_override is None else _c(pos_override, np.int32)
        pos_all[ti] = pos
        kk = keys(codes, seq_off, l, pos)
        if with_counts:
            cnts.append(counts(kk, k))
        a, b, o, m = enriched(kk, s)
        ct.append(np.full(a.size, trial, np.int32)); ck.append(a); cc.append(b)
        offs.append(o[1:] + base); mems.append(m)
        base += m.size
    out = {
        "positions": pos_all,
        "cand_trial": np.concatenate(ct) if ct else np.zeros(0, np.int32),
        "cand_key": np.concatenate(ck) if ck else np.zeros(0, np.uint32),
        "cand_cnt": np.concatenate(cc) if cc else np.zeros(0, np.int32),
        "cand_off": np.concatenate([np.array([0], np.int64)] + offs).astype(np.int64),
        "members": np.concatenate(mems) if mems else np.zeros(0, np.int32),
    }
    if with_counts:
        out["counts"] = np.stack(cnts) if cnts else np.zeros((0, 4 ** k), np.uint32)
    return out


# --------------------------------------------------------------------------
# Section 5 parameter choice
# --------------------------------------------------------------------------

def m_bound(l, d, k, s, t_hat, q=0.95) -> int:
    return int(_L().orc_m_bound(l, d, k, s, t_hat, q))


def default_params(lens, l, d, k=0, s=0, m=0, q=0.95):
    """Algorithm 2 step 1 ("if not specified"): k = l-d-1; s = max(3, ceil(2x/4^k))
    (twice the mean bucket size, floored at the paper's empirical 3);
    m = the Section 5 bound at probability q with t_hat = t."""
    lens = [int(n) for n in lens]
    x = sum(max(0, n - l + 1) for n in lens)
    if k == 0:
        k = l - d - 1
    if s == 0:
        s = max(3, math.ceil(2.0 * x / 4.0 ** k))
    if m == 0:
        m = m_bound(l, d, k, s, len(lens), q)
    return k, s, m


# --------------------------------------------------------------------------
# Section 5.1: theta^0, EM, sites, consensus, Score
# --------------------------------------------------------------------------

def background(codes) -> np.ndarray:
    codes = _c(codes, np.uint8)
    bg = np.empty(4, np.float64)
    _L().orc_background(_p(codes), codes.size, _p(bg))
    return bg


def theta0(codes, seq_off, l, members, beta) -> np.ndarray:
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64); members = _c(members, np.int32)
    lo = lmer_offsets(seq_off, l)
    pwm = np.empty((l, 4), np.float64)
    _L().orc_theta0(_p(codes), _p(seq_off), _p(lo), seq_off.size - 1, l, _p(members),
                    members.size, float(beta), _p(pwm))
    return pwm


def theta0_all(codes, seq_off, l, cand_off, members, beta) -> np.ndarray:
    C = len(cand_off) - 1
    out = np.empty((C, l, 4), np.float64)
    for c in range(C):
        out[c] = theta0(codes, seq_off, l, members[cand_off[c]:cand_off[c + 1]], beta)
    return out


def em(codes, seq_off, l, bg, pwm0, iters, beta, want_lse=False, want_trace=False, nthreads=1):
    """OOPS EM from each starting model pwm0[C][l][4]: returns (pwm, ll[, lse][, trace])."""
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64)
    pwm = np.array(pwm0, dtype=np.float64, copy=True, order="C").reshape(-1, l, 4)
    C = pwm.shape[0]
    t = seq_off.size - 1
    bg = _c(bg, np.float64)
    ll = np.empty(C, np.float64)
    lse = np.empty((C, t), np.float64) if want_lse else None
    tr = np.empty((C, iters + 1), np.float64) if want_trace else None
    rc = _L().orc_em(_p(codes), _p(seq_off), t, l, _p(bg), _p(pwm), C, iters, float(beta),
                     _p(ll), _p(lse), _p(tr), int(nthreads))
    if rc != 0:
        raise ValueError("bad EM arguments")
    out = [pwm, ll]
    if want_lse:
        out.append(lse)
    if want_trace:
        out.append(tr)
    return tuple(out)


def em_zoops(codes, seq_off, l, bg, pwm0, iters, beta, gamma, want_trace=False, nthreads=1):
    """ZOOPS EM (site probability gamma per sequence) from each starting model
    pwm0[C][l][4]: returns (pwm, ll[, trace])."""
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64)
    pwm = np.array(pwm0, dtype=np.float64, copy=True, order="C").reshape(-1, l, 4)
    C = pwm.shape[0]
    t = seq_off.size - 1
    bg = _c(bg, np.float64)
    ll = np.empty(C, np.float64)
    tr = np.empty((C, iters + 1), np.float64) if want_trace else None
    rc = _L().orc_em_zoops(_p(codes), _p(seq_off), t, l, _p(bg), _p(pwm), C, iters, float(beta),
                           float(gamma), _p(ll), _p(tr), int(nthreads))
    if rc != 0:
        raise ValueError("bad EM arguments")
    return (pwm, ll, tr) if want_trace else (pwm, ll)


def sites(codes, seq_off, l, bg, pwm) -> np.ndarray:
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64)
    pwm = _c(pwm, np.float64); bg = _c(bg, np.float64)
    t = seq_off.size - 1
    out = np.empty(t, np.int32)
    _L().orc_sites(_p(codes), _p(seq_off), t, l, _p(bg), _p(pwm), _p(out))
    return out


def consensus(pwm) -> str:
    pwm = _c(pwm, np.float64)
    l = pwm.shape[0]
    buf = ctypes.create_string_buffer(l + 1)
    _L().orc_consensus(_p(pwm), l, buf)
    return buf.value.decode()


def score(codes, seq_off, l, sites_) -> int:
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64); sites_ = _c(sites_, np.int32)
    return int(_L().orc_score(_p(codes), _p(seq_off), seq_off.size - 1, l, _p(sites_)))


def top_candidates(cand_cnt, top: int) -> np.ndarray:
    """The `top` candidates with the most member l-mers, in that order; equal
    counts keep the (trial, key) order of the candidate list.  Reading of the
    "top 1024 enriched buckets" of the serving-scale workload: the paper ranks
    buckets only by the threshold s (Algorithm 2 step 3), so a cap on their
    number keeps the largest buckets."""
    cnt = np.asarray(cand_cnt, np.int64)
    order = np.lexsort((np.arange(cnt.size), -cnt))
    return order[:top].astype(np.int64)


def rank(ll: np.ndarray) -> int:
    """Best candidate: the highest log-likelihood ratio; a tie goes to the
    candidate that comes first in (trial, key) order."""
    ll = np.asarray(ll, np.float64)
    return int(np.argmax(ll)) if ll.size else -1


def find(ascii_seqs, l, d, k=0, s=0, m=0, seed=0, em_iters=5, beta=0.25, nthreads=1,
         subset=None, with_hash=False, top=0):
    """Whole pipeline (Algorithm 2 + Section 5.1) on a list of ASCII sequences.

    ``subset``: optional candidate indices; EM then runs on those candidates
    only (used to bound the oracle's cost on large inputs)."""
    lens = [len(q) for q in ascii_seqs]
    seq_off = np.zeros(len(lens) + 1, np.int64)
    seq_off[1:] = np.cumsum(lens)
    codes = encode(b"".join(bytes(q, "ascii") if isinstance(q, str) else bytes(q)
                            for q in ascii_seqs))
    k, s, m = default_params(lens, l, d, k, s, m)
    h = hash_trials(codes, seq_off, l, k, s, seed, 0, m)
    C = h["cand_key"].size
    if top and C > top:
        idx = top_candidates(h["cand_cnt"], top)
    else:
        idx = np.arange(C) if subset is None else np.asarray(subset, np.int64)
    bg = background(codes)
    th0 = np.empty((idx.size, l, 4))
    for n, c in enumerate(idx):
        th0[n] = theta0(codes, seq_off, l, h["members"][h["cand_off"][c]:h["cand_off"][c + 1]], beta)
    pwm, ll = em(codes, seq_off, l, bg, th0, em_iters, beta, nthreads=nthreads)
    res = {"k": k, "s": s, "m": m, "n_candidates": C, "bg": bg, "cand_index": idx,
           "pwm_all": pwm, "ll_all": ll}
    if idx.size:
        b = rank(ll)
        w = int(idx[b])
        st = sites(codes, seq_off, l, bg, pwm[b])
        res.update(win=w, win_trial=int(h["cand_trial"][w]), win_key=int(h["cand_key"][w]),
                   pwm=pwm[b], loglik=float(ll[b]), consensus=consensus(pwm[b]), sites=st,
                   score=score(codes, seq_off, l, st))
    if with_hash:
        res["hash"] = h
    return res


# --------------------------------------------------------------------------
# Protein alphabet (reading R17): 20 letters ACDEFGHIKLMNPQRSTVWY, codes 0..19
# --------------------------------------------------------------------------

AA_LETTERS = "ACDEFGHIKLMNPQRSTVWY"


def encode_aa(ascii_bytes) -> np.ndarray:
    a = np.frombuffer(bytes(ascii_bytes), np.uint8)
    out = np.empty(a.size, np.uint8)
    bad = _L().orc_encode_aa(_p(a), a.size, _p(out))
    if bad >= 0:
        raise ValueError(f"not an amino-acid letter at {bad}")
    return out


def keys_a(codes, seq_off, l, pos, A):
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64); pos = _c(pos, np.int32)
    t = seq_off.size - 1
    x = int(np.sum(np.maximum(np.diff(seq_off) - l + 1, 0)))
    out = np.empty(x, np.uint32)
    _L().orc_keys_a(_p(codes), _p(seq_off), t, l, pos.size, _p(pos), A, _p(out))
    return out


def background_a(codes, A) -> np.ndarray:
    codes = _c(codes, np.uint8)
    bg = np.empty(A, np.float64)
    _L().orc_background_a(_p(codes), codes.size, A, _p(bg))
    return bg


def theta0_a(codes, seq_off, l, members, beta, A) -> np.ndarray:
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64)
    lo = lmer_offsets(seq_off, l)
    mem = _c(members, np.int32)
    out = np.empty((l, A), np.float64)
    _L().orc_theta0_a(_p(codes), _p(seq_off), _p(lo), seq_off.size - 1, l, _p(mem), mem.size,
                      float(beta), A, _p(out))
    return out


def em_a(codes, seq_off, l, bg, pwm0, iters, beta, A, nthreads=1):
    """OOPS EM over an alphabet of A letters from pwm0[C][l][A]: (pwm, ll)."""
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64)
    pwm = np.array(pwm0, dtype=np.float64, copy=True, order="C").reshape(-1, l, A)
    C = pwm.shape[0]
    bg = _c(bg, np.float64)
    ll = np.empty(C, np.float64)
    rc = _L().orc_em_a(_p(codes), _p(seq_off), seq_off.size - 1, l, A, _p(bg), _p(pwm), C, iters,
                       float(beta), _p(ll), int(nthreads))
    if rc != 0:
        raise ValueError("bad EM arguments")
    return pwm, ll


def sites_a(codes, seq_off, l, bg, pwm, A) -> np.ndarray:
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64)
    pwm = _c(pwm, np.float64); bg = _c(bg, np.float64)
    out = np.empty(seq_off.size - 1, np.int32)
    _L().orc_sites_a(_p(codes), _p(seq_off), seq_off.size - 1, l, A, _p(bg), _p(pwm), _p(out))
    return out


def consensus_a(pwm, A, letters=AA_LETTERS) -> str:
    pwm = _c(pwm, np.float64)
    l = pwm.size // A
    buf = ctypes.create_string_buffer(l + 1)
    _L().orc_consensus_a(_p(pwm), l, A, letters.encode(), buf)
    return buf.value.decode()


def score_a(codes, seq_off, l, sites, A) -> int:
    codes = _c(codes, np.uint8); seq_off = _c(seq_off, np.int64); sites = _c(sites, np.int32)
    return int(_L().orc_score_a(_p(codes), _p(seq_off), seq_off.size - 1, l, A, _p(sites)))


def find_protein(seqs, l, k, s, m, seed, em_iters, beta, nthreads=1):
    """Algorithm 2 + Section 5.1 over the 20-letter alphabet (keys base 20,
    enriched buckets by grouping equal keys, OOPS EM on every candidate)."""
    A = 20
    codes = encode_aa(b"".join(bytes(q, "ascii") if isinstance(q, str) else bytes(q) for q in seqs))
    seq_off = np.concatenate([[0], np.cumsum([len(q) for q in seqs])]).astype(np.int64)
    ct, ck, cc, offs, mems, base = [], [], [], [], [], 0
    for trial in range(m):
        kk = keys_a(codes, seq_off, l, positions(seed, trial, l, k), A)
        a, b, o, mm = enriched(kk, s)
        ct.append(np.full(a.size, trial, np.int32)); ck.append(a); cc.append(b)
        offs.append(o[1:] + base); mems.append(mm)
        base += mm.size
    cand_off = np.concatenate([np.array([0], np.int64)] + offs).astype(np.int64)
    members = np.concatenate(mems) if mems else np.zeros(0, np.int32)
    C = int(cand_off.size - 1)
    res = {"k": k, "s": s, "m": m, "n_candidates": C,
           "cand_trial": np.concatenate(ct) if ct else np.zeros(0, np.int32),
           "cand_key": np.concatenate(ck) if ck else np.zeros(0, np.uint32),
           "cand_cnt": np.concatenate(cc) if cc else np.zeros(0, np.int32),
           "cand_off": cand_off, "members": members}
    if C == 0:
        return res
    bg = background_a(codes, A)
    th0 = np.stack([theta0_a(codes, seq_off, l, members[cand_off[c]:cand_off[c + 1]], beta, A)
                    for c in range(C)])
    pwm, ll = em_a(codes, seq_off, l, bg, th0, em_iters, beta, A, nthreads=nthreads)
    w = rank(ll)
    st = sites_a(codes, seq_off, l, bg, pwm[w], A)
    res.update(bg=bg, pwm_all=pwm, ll_all=ll, win=w, pwm=pwm[w], loglik=float(ll[w]),
               consensus=consensus_a(pwm[w], A), sites=st, score=score_a(codes, seq_off, l, st, A))
    return res
