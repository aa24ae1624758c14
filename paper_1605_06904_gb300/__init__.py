"""GB300 (sm_103a) PROJECTION motif finder -- Python binding of include/projection.h.

Every step of the method runs in the CUDA library ``libprojection.so``; this
module only marshals arguments.  PyTorch provides device memory and the
current stream.  Function names follow the C ABI.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import (PROJ_EM_BF16_SPLIT, PROJ_EM_FP32, ProjectionError,  # noqa: F401
                      ProjectionResult, check, lib)

__all__ = ["projection_packed_words", "projection_default_params", "projection_pack",
           "projection_background", "projection_positions", "trial_hash",
           "trial_hash_noalloc", "trial_hash_top", "theta0_build",
           "em_refine", "projection_finalize", "projection_find", "projection_find_packed",
           "projection_find_batch", "projection_find_top", "projection_find_protein", "projection_find_packed_top",
           "projection_trace_enable", "projection_trace_read", "projection_selftest_wait",
           "projection_hist_peak", "projection_ex2_peak", "projection_params_batch", "em_refine_zoops",
           "projection_find_packed_zoops", "trial_hash_allpairs", "ProjectionError",
           "PROJ_EM_FP32", "PROJ_EM_BF16_SPLIT", "seq_offsets"]


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dev(n, dtype, device):
    return torch.empty(int(n), dtype=dtype, device=device)


def seq_offsets(lens) -> np.ndarray:
    lens = np.asarray(lens, np.int64)
    off = np.zeros(lens.size + 1, np.int64)
    off[1:] = np.cumsum(lens)
    return off


def _off(seq_off) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq_off, dtype=np.int64))


# ---- host helpers ----------------------------------------------------------

def projection_packed_words(total_bases: int) -> int:
    return int(lib().projection_packed_words(int(total_bases)))


def projection_default_params(lens, l, d, k=0, s=0, m=0):
    lens = np.ascontiguousarray(np.asarray(lens, np.int64))
    K, S, M = ctypes.c_int(k), ctypes.c_int(s), ctypes.c_int(m)
    check(lib().projection_default_params(lens.size, _ptr(lens), l, d, ctypes.byref(K),
                                          ctypes.byref(S), ctypes.byref(M)))
    return K.value, S.value, M.value


# ---- steps -------------------------------------------------------------------

def projection_pack(ascii_dev: torch.Tensor, stream=None) -> torch.Tensor:
    """uint8 CUDA tensor of ASCII bases -> int32 tensor of packed 2-bit words.
    Raises ProjectionError(PROJ_EBADCHAR) naming the first non-ACGT index."""
    assert ascii_dev.dtype == torch.uint8 and ascii_dev.is_contiguous()
    n = ascii_dev.numel()
    packed = _dev(max(1, projection_packed_words(n)), torch.int32, ascii_dev.device)
    bad = _dev(1, torch.int64, ascii_dev.device)
    check(lib().projection_pack(_ptr(ascii_dev), n, _ptr(packed), _ptr(bad), _stream(stream)))
    b = int(bad.item())
    if b >= 0:
        raise ProjectionError(_native.PROJ_EBADCHAR, f"character at index {b} is not A/C/G/T")
    return packed


def projection_background(packed: torch.Tensor, total_bases: int, stream=None) -> torch.Tensor:
    bg = _dev(4, torch.float64, packed.device)
    check(lib().projection_background(_ptr(packed), int(total_bases), _ptr(bg), _stream(stream)))
    return bg


def projection_positions(seed, trial_begin, n_trials, l, k, device="cuda", stream=None):
    pos = _dev(max(1, n_trials * k), torch.uint8, device)
    check(lib().projection_positions(seed & (2**64 - 1), trial_begin, n_trials, l, k, _ptr(pos),
                                     _stream(stream)))
    return pos[:n_trials * k].view(n_trials, k)


def trial_hash(packed, seq_off, l, k, s, seed, trial_begin, n_trials, positions_in=None,
               want_positions=False, want_counts=False, cap_cand=None, cap_members=None,
               stream=None):
    """Algorithm 2 steps 2-3 for trials [trial_begin, trial_begin + n_trials).
    Returns a dict of CUDA tensors: cand_trial, cand_key (int32 storage of
    uint32), cand_cnt, cand_off, members, and optionally positions and counts."""
    off = _off(seq_off)
    t = off.size - 1
    dev = packed.device
    x = int(np.sum(np.maximum(np.diff(off) - l + 1, 0)))
    if cap_members is None:
        cap_members = max(1, min(x * n_trials, 1 << 26))
    if cap_cand is None:
        cap_cand = max(1, cap_members // max(1, s))
    pin = None
    if positions_in is not None:
        pin = np.ascontiguousarray(np.asarray(positions_in, np.int32))
        assert pin.size == k
    pos = _dev(max(1, n_trials * k), torch.uint8, dev) if want_positions else None
    cnt = _dev(max(1, n_trials * 4 ** k), torch.int32, dev) if want_counts else None
    while True:
        ct = _dev(cap_cand, torch.int32, dev)
        ck = _dev(cap_cand, torch.int32, dev)
        cc = _dev(cap_cand, torch.int32, dev)
        co = _dev(cap_cand + 1, torch.int64, dev)
        mem = _dev(cap_members, torch.int32, dev)
        tot = _dev(2, torch.int64, dev)
        check(lib().trial_hash(_ptr(packed), _ptr(off), t, l, k, s, seed & (2**64 - 1),
                               trial_begin, n_trials, _ptr(pin), _ptr(pos), _ptr(cnt), cap_cand,
                               cap_members, _ptr(ct), _ptr(ck), _ptr(cc), _ptr(co), _ptr(mem),
                               _ptr(tot), _stream(stream)))
        C, M = (int(v) for v in tot.cpu())
        if C <= cap_cand and M <= cap_members:
            break
        cap_cand, cap_members = max(C, 1), max(M, 1)
    out = {"cand_trial": ct[:C], "cand_key": ck[:C], "cand_cnt": cc[:C], "cand_off": co[:C + 1],
           "members": mem[:M], "n_candidates": C, "n_members": M}
    if want_positions:
        out["positions"] = pos[:n_trials * k].view(n_trials, k)
    if want_counts:
        out["counts"] = cnt[:n_trials * 4 ** k].view(n_trials, 4 ** k)
    return out


def trial_hash_top(packed, seq_off, l, k, s, seed, n_trials, top, cap_members=None, stream=None):
    """Algorithm 2 steps 2-3 for trials [0, n_trials), keeping the `top` largest
    enriched buckets (size descending, ties in (trial, key) order).  Returns a
    dict of CUDA tensors sel_index, cand_trial, cand_key (int32 storage of
    uint32), cand_cnt, cand_off, members, and the totals."""
    off = _off(seq_off)
    t = off.size - 1
    dev = packed.device
    if cap_members is None:
        cap_members = max(1, 64 * top)
    while True:
        si = _dev(top, torch.int64, dev)
        ct = _dev(top, torch.int32, dev)
        ck = _dev(top, torch.int32, dev)
        cc = _dev(top, torch.int32, dev)
        co = _dev(top + 1, torch.int64, dev)
        mem = _dev(cap_members, torch.int32, dev)
        tot = _dev(4, torch.int64, dev)
        rc = lib().trial_hash_top(_ptr(packed), _ptr(off), t, l, k, s, seed & (2**64 - 1), n_trials,
                                  top, cap_members, _ptr(si), _ptr(ct), _ptr(ck), _ptr(cc),
                                  _ptr(co), _ptr(mem), _ptr(tot), _stream(stream))
        if rc == _native.PROJ_ECAPACITY:
            cap_members = int(tot.cpu()[3])
            continue
        check(rc)
        break
    C, M, R, K = (int(v) for v in tot.cpu())
    return {"sel_index": si[:R], "cand_trial": ct[:R], "cand_key": ck[:R], "cand_cnt": cc[:R],
            "cand_off": co[:R + 1], "members": mem[:K], "n_candidates": C, "n_members": M,
            "n_kept": R, "kept_members": K}


def trial_hash_allpairs(packed, seq_off, l, k, s, seed, trial_begin, n_trials, cap_cand=None,
                        cap_members=None, stream=None):
    """trial_hash's output from the low-memory all-pairs mode (no 4^k table;
    O(x^2) comparisons per trial)."""
    off = _off(seq_off)
    t = off.size - 1
    dev = packed.device
    x = int(np.sum(np.maximum(np.diff(off) - l + 1, 0)))
    if cap_members is None:
        cap_members = max(1, min(x * n_trials, 1 << 26))
    if cap_cand is None:
        cap_cand = max(1, cap_members // max(1, s))
    while True:
        ct = _dev(cap_cand, torch.int32, dev)
        ck = _dev(cap_cand, torch.int32, dev)
        cc = _dev(cap_cand, torch.int32, dev)
        co = _dev(cap_cand + 1, torch.int64, dev)
        mem = _dev(cap_members, torch.int32, dev)
        tot = _dev(2, torch.int64, dev)
        check(lib().trial_hash_allpairs(_ptr(packed), _ptr(off), t, l, k, s, seed & (2**64 - 1),
                                        trial_begin, n_trials, cap_cand, cap_members, _ptr(ct),
                                        _ptr(ck), _ptr(cc), _ptr(co), _ptr(mem), _ptr(tot),
                                        _stream(stream)))
        C, M = (int(v) for v in tot.cpu())
        if C <= cap_cand and M <= cap_members:
            break
        cap_cand, cap_members = max(C, 1), max(M, 1)
    return {"cand_trial": ct[:C], "cand_key": ck[:C], "cand_cnt": cc[:C], "cand_off": co[:C + 1],
            "members": mem[:M], "n_candidates": C, "n_members": M}


def trial_hash_noalloc(packed, seq_off, l, k, s, seed, trial_begin, n_trials, cap_cand,
                       cap_members, positions_in=None, stream=None):
    """trial_hash without device allocation inside the library (scratch in a
    fixed array of PROJ_NOALLOC_SCRATCH_BYTES).  Output tensors are
    allocated here, by the caller side, with fixed capacities; raises
    ProjectionError(PROJ_ECAPACITY) when the scratch or a capacity is too
    small."""
    off = _off(seq_off)
    t = off.size - 1
    dev = packed.device
    pin = None
    if positions_in is not None:
        pin = np.ascontiguousarray(np.asarray(positions_in, np.int32))
    ct = _dev(max(1, cap_cand), torch.int32, dev)
    ck = _dev(max(1, cap_cand), torch.int32, dev)
    cc = _dev(max(1, cap_cand), torch.int32, dev)
    co = _dev(cap_cand + 1, torch.int64, dev)
    mem = _dev(max(1, cap_members), torch.int32, dev)
    tot = _dev(2, torch.int64, dev)
    check(lib().trial_hash_noalloc(_ptr(packed), _ptr(off), t, l, k, s, seed & (2**64 - 1),
                                   trial_begin, n_trials, _ptr(pin), None, None, cap_cand,
                                   cap_members, _ptr(ct), _ptr(ck), _ptr(cc), _ptr(co), _ptr(mem),
                                   _ptr(tot), _stream(stream)))
    C, M = (int(v) for v in tot.cpu())
    if C > cap_cand or M > cap_members:
        raise ProjectionError(_native.PROJ_ECAPACITY,
                              f"need {C} candidates / {M} members, capacities {cap_cand} / {cap_members}")
    return {"cand_trial": ct[:C], "cand_key": ck[:C], "cand_cnt": cc[:C], "cand_off": co[:C + 1],
            "members": mem[:M], "n_candidates": C, "n_members": M}


def theta0_build(packed, seq_off, l, cand_off, members, C, pseudocount, stream=None):
    off = _off(seq_off)
    th = _dev(max(1, C * l * 4), torch.float32, packed.device)
    check(lib().theta0_build(_ptr(packed), _ptr(off), off.size - 1, l, _ptr(cand_off),
                             _ptr(members), C, float(pseudocount), _ptr(th), _stream(stream)))
    return th[:C * l * 4].view(C, l, 4)


def em_refine(packed, seq_off, l, bg, theta0, em_iters, pseudocount, precision=PROJ_EM_FP32,
              out=None, stream=None, want_sites=False):
    """OOPS EM (Section 5.1) from theta0 [C, l, 4] (float32 CUDA).  Returns
    (theta [C, l, 4] float32, loglik [C] float64), plus sites [C, t] int32
    (Definition 1's start vector under each final model) with want_sites."""
    off = _off(seq_off)
    C = theta0.shape[0]
    t = off.size - 1
    theta0 = theta0.contiguous()
    th = torch.empty_like(theta0) if out is None else out
    ll = _dev(max(1, C), torch.float64, theta0.device)
    sites = _dev(max(1, C * t), torch.int32, theta0.device) if want_sites else None
    check(lib().em_refine(_ptr(packed), _ptr(off), t, l, _ptr(bg), _ptr(theta0), C,
                          em_iters, float(pseudocount), precision, _ptr(th), _ptr(ll),
                          _ptr(sites), _stream(stream)))
    if want_sites:
        return th, ll[:C], sites[:C * t].view(C, t)
    return th, ll[:C]


def projection_finalize(packed, seq_off, l, bg, theta, loglik, stream=None):
    off = _off(seq_off)
    t = off.size - 1
    dev = packed.device
    C = theta.shape[0]
    best = _dev(1, torch.int64, dev)
    sites = _dev(t, torch.int32, dev)
    cons = _dev(l, torch.uint8, dev)
    score = _dev(1, torch.int32, dev)
    check(lib().projection_finalize(_ptr(packed), _ptr(off), t, l, _ptr(bg), _ptr(theta),
                                    _ptr(loglik), C, _ptr(best), _ptr(sites), _ptr(cons),
                                    _ptr(score), _stream(stream)))
    return {"best": int(best.item()), "sites": sites.cpu().numpy(),
            "consensus": bytes(cons.cpu().numpy()).decode(), "score": int(score.item())}


def _result_dict(r: ProjectionResult, alphabet: int = 4) -> dict:
    l, t = r.l, r.t
    out = {"status": r.status, "t": t, "l": l, "k": r.k, "s": r.s, "m": r.m,
           "n_candidates": r.n_candidates, "n_members": r.n_members, "win_index": r.win_index,
           "win_trial": r.win_trial, "win_key": r.win_key, "loglik": r.loglik,
           "score": r.score, "n_refined": r.n_refined}
    if r.pwm:
        out["pwm"] = np.ctypeslib.as_array(r.pwm, shape=(l * alphabet,)).reshape(l, alphabet).copy()
        out["sites"] = np.ctypeslib.as_array(r.sites, shape=(t,)).copy()
        out["consensus"] = r.consensus.decode()
    return out


def projection_find(ascii, seq_off, l, d, k=0, s=0, m=0, seed=0, em_iters=5, pseudocount=0.25,
                    precision=PROJ_EM_FP32, stream=None) -> dict:
    """Whole path from HOST sequences in linear form (uint8 ASCII array +
    int64 offsets).  The input may be pinned (torch CPU tensor) or numpy."""
    off = _off(seq_off)
    if isinstance(ascii, torch.Tensor):
        assert ascii.device.type == "cpu" and ascii.dtype == torch.uint8
        aptr = ctypes.c_void_p(ascii.data_ptr())
    else:
        ascii = np.ascontiguousarray(np.asarray(ascii, np.uint8))
        aptr = _ptr(ascii)
    r = ProjectionResult()
    rc = lib().projection_find(aptr, _ptr(off), off.size - 1, l, d, k, s, m, seed & (2**64 - 1),
                               em_iters, float(pseudocount), precision, ctypes.byref(r),
                               _stream(stream))
    try:
        check(rc)
        return _result_dict(r)
    finally:
        lib().projection_result_free(ctypes.byref(r))


def projection_find_top(ascii, seq_off, l, d, k=0, s=0, m=0, seed=0, em_iters=5,
                        pseudocount=0.25, precision=PROJ_EM_FP32, top=0, stream=None) -> dict:
    """projection_find refining only the `top` largest enriched buckets."""
    off = _off(seq_off)
    ascii = np.ascontiguousarray(np.asarray(ascii, np.uint8))
    r = ProjectionResult()
    rc = lib().projection_find_top(_ptr(ascii), _ptr(off), off.size - 1, l, d, k, s, m,
                                   seed & (2**64 - 1), em_iters, float(pseudocount), precision,
                                   int(top), ctypes.byref(r), _stream(stream))
    try:
        check(rc)
        return _result_dict(r)
    finally:
        lib().projection_result_free(ctypes.byref(r))


def projection_find_protein(ascii, seq_off, l, k, s, m, seed=0, em_iters=5, pseudocount=0.25,
                            stream=None) -> dict:
    """Algorithm 2 + OOPS EM over the 20 amino-acid letters from HOST ASCII
    sequences in linear form; the result's "pwm" is [l, 20]."""
    off = _off(seq_off)
    ascii = np.ascontiguousarray(np.asarray(ascii, np.uint8))
    r = ProjectionResult()
    rc = lib().projection_find_protein(_ptr(ascii), _ptr(off), off.size - 1, l, k, s, m,
                                       seed & (2**64 - 1), em_iters, float(pseudocount),
                                       ctypes.byref(r), _stream(stream))
    try:
        check(rc)
        return _result_dict(r, 20)
    finally:
        lib().projection_result_free(ctypes.byref(r))


def em_refine_zoops(packed, seq_off, l, bg, theta0, em_iters, pseudocount, site_prob,
                    precision=PROJ_EM_FP32, out=None, stream=None, want_sites=False):
    """ZOOPS EM (site probability `site_prob` per sequence) from theta0 [C, l, 4]
    (float32 CUDA).  Returns (theta [C, l, 4] float32, loglik [C] float64), plus
    sites [C, t] int32 with want_sites."""
    off = _off(seq_off)
    C = theta0.shape[0]
    t = off.size - 1
    theta0 = theta0.contiguous()
    th = torch.empty_like(theta0) if out is None else out
    ll = _dev(max(1, C), torch.float64, theta0.device)
    sites = _dev(max(1, C * t), torch.int32, theta0.device) if want_sites else None
    check(lib().em_refine_zoops(_ptr(packed), _ptr(off), t, l, _ptr(bg), _ptr(theta0),
                                C, em_iters, float(pseudocount), precision, float(site_prob),
                                _ptr(th), _ptr(ll), _ptr(sites), _stream(stream)))
    if want_sites:
        return th, ll[:C], sites[:C * t].view(C, t)
    return th, ll[:C]


def projection_find_packed_zoops(packed, seq_off, l, d, k=0, s=0, m=0, seed=0, em_iters=5,
                                 pseudocount=0.25, precision=PROJ_EM_FP32, site_prob=0.5, top=0,
                                 stream=None) -> dict:
    off = _off(seq_off)
    r = ProjectionResult()
    rc = lib().projection_find_packed_zoops(_ptr(packed), _ptr(off), off.size - 1, l, d, k, s, m,
                                            seed & (2**64 - 1), em_iters, float(pseudocount),
                                            precision, float(site_prob), int(top), ctypes.byref(r),
                                            _stream(stream))
    try:
        check(rc)
        return _result_dict(r)
    finally:
        lib().projection_result_free(ctypes.byref(r))


def projection_find_packed_top(packed, seq_off, l, d, k=0, s=0, m=0, seed=0, em_iters=5,
                               pseudocount=0.25, precision=PROJ_EM_FP32, top=0,
                               stream=None) -> dict:
    off = _off(seq_off)
    r = ProjectionResult()
    rc = lib().projection_find_packed_top(_ptr(packed), _ptr(off), off.size - 1, l, d, k, s, m,
                                          seed & (2**64 - 1), em_iters, float(pseudocount),
                                          precision, int(top), ctypes.byref(r), _stream(stream))
    try:
        check(rc)
        return _result_dict(r)
    finally:
        lib().projection_result_free(ctypes.byref(r))


def projection_find_packed(packed, seq_off, l, d, k=0, s=0, m=0, seed=0, em_iters=5,
                           pseudocount=0.25, precision=PROJ_EM_FP32, stream=None) -> dict:
    off = _off(seq_off)
    r = ProjectionResult()
    rc = lib().projection_find_packed(_ptr(packed), _ptr(off), off.size - 1, l, d, k, s, m,
                                      seed & (2**64 - 1), em_iters, float(pseudocount), precision,
                                      ctypes.byref(r), _stream(stream))
    try:
        check(rc)
        return _result_dict(r)
    finally:
        lib().projection_result_free(ctypes.byref(r))


def projection_find_batch(instances, l, d, k=None, s=None, m=None, seeds=None, em_iters=5,
                          pseudocount=0.25, precision=PROJ_EM_BF16_SPLIT, stream=None) -> list:
    """Many independent searches in one call.  `instances` is a list of
    instances, each a list of ASCII sequences (bytes); l, d, k, s, m, seeds are
    per-instance sequences (k, s, m may be None or contain 0 = Section 5
    choice).  Returns one result dict per instance."""
    n = len(instances)
    seqs = [q for inst in instances for q in inst]
    ascii = np.frombuffer(b"".join(bytes(q) for q in seqs), dtype=np.uint8)
    off = seq_offsets([len(q) for q in seqs])
    inst_seq = np.zeros(n + 1, np.int32)
    inst_seq[1:] = np.cumsum([len(inst) for inst in instances])
    arr = lambda v, dt, dflt: np.ascontiguousarray(np.asarray(v if v is not None else [dflt] * n, dt))
    L, D = arr(l, np.int32, 0), arr(d, np.int32, 0)
    K, S, M = arr(k, np.int32, 0), arr(s, np.int32, 0), arr(m, np.int32, 0)
    SE = np.ascontiguousarray(np.asarray(seeds if seeds is not None else np.arange(n), np.uint64))
    res = (ProjectionResult * n)()
    rc = lib().projection_find_batch(_ptr(ascii), _ptr(off), _ptr(inst_seq), n, _ptr(L), _ptr(D),
                                     _ptr(K), _ptr(S), _ptr(M), _ptr(SE), em_iters,
                                     float(pseudocount), precision, res, _stream(stream))
    try:
        check(rc)
        return [_result_dict(r) for r in res]
    finally:
        for i in range(n):
            lib().projection_result_free(ctypes.byref(res[i]))


def projection_selftest_wait(timeout_ns: int = 50_000_000, stream=None) -> int:
    """Runs the bounded-wait self-test; returns the status (PROJ_ETIMEOUT = -5
    is the expected one)."""
    return int(lib().projection_selftest_wait(int(timeout_ns), _stream(stream)))


def projection_params_batch(t, x, l, d, k=None, s=None, m=None, q=0.95, stream=None):
    """Algorithm 2 step 1 for a batch on the device (Section 5).  t, l, d, k, s,
    m: int32 CUDA tensors [n] (k, s, m optional: zeros = derive); x: int64 CUDA
    tensor [n] of l-mer counts.  Returns (k, s, m, status) as CUDA tensors."""
    n = int(t.numel())
    dev = t.device
    z = lambda: torch.zeros(n, dtype=torch.int32, device=dev)
    k = (k if k is not None else z()).to(torch.int32).contiguous().clone()
    s = (s if s is not None else z()).to(torch.int32).contiguous().clone()
    m = (m if m is not None else z()).to(torch.int32).contiguous().clone()
    status = z()
    t, x, l, d = (v.contiguous() for v in (t.to(torch.int32), x.to(torch.int64),
                                           l.to(torch.int32), d.to(torch.int32)))
    check(lib().projection_params_batch(n, _ptr(t), _ptr(x), _ptr(l), _ptr(d), _ptr(k), _ptr(s),
                                        _ptr(m), _ptr(status), float(q), _stream(stream)))
    return k, s, m, status


def projection_hist_peak(k: int, stream=None) -> float:
    """Shared-memory histogram increments per second for 4^k buckets (the
    bucket kernels' roofline denominator)."""
    out = ctypes.c_double(0.0)
    check(lib().projection_hist_peak(int(k), ctypes.byref(out), _stream(stream)))
    return float(out.value)


def projection_ex2_peak(stream=None) -> float:
    """exp2 (ex2.approx) evaluations per second on this GPU (the EM kernels'
    exponential roofline denominator)."""
    out = ctypes.c_double(0.0)
    check(lib().projection_ex2_peak(ctypes.byref(out), _stream(stream)))
    return float(out.value)


# ---- tracing -----------------------------------------------------------------

def projection_trace_enable(on: bool = True) -> None:
    check(lib().projection_trace_enable(1 if on else 0))


def projection_trace_read(prefix: str = ""):
    """(summed device milliseconds, launches) of the traced kernels whose name
    starts with `prefix`."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    check(lib().projection_trace_read(prefix.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value
