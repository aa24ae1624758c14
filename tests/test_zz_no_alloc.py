"""trial_hash_noalloc: the hashing entry point for callers that cannot allocate
device memory (a service whose memory all belongs to its own pool allocator, or
a latency-critical path that must not pay for an allocation).  It must give
exactly what trial_hash gives -- bucket lists are integer data, so bit for bit
-- on consecutive calls that reuse its fixed scratch array, and must refuse
work that does not fit that array instead of launching it.

The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from synth import instance_for_config

pytestmark = pytest.mark.gpu


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else None


def _noalloc(lib, packed, off, l, k, s, seed, t0, T, cap_c, cap_m):
    """One call of the C entry point with caller-owned output buffers."""
    dev = packed.device
    out = {
        "cand_trial": torch.full((cap_c,), -1, dtype=torch.int32, device=dev),
        "cand_key": torch.full((cap_c,), -1, dtype=torch.int32, device=dev),
        "cand_cnt": torch.full((cap_c,), -1, dtype=torch.int32, device=dev),
        "cand_off": torch.full((cap_c + 1,), -1, dtype=torch.int64, device=dev),
        "members": torch.full((cap_m,), -1, dtype=torch.int32, device=dev),
    }
    tot = torch.zeros(2, dtype=torch.int64, device=dev)
    off = np.ascontiguousarray(off, np.int64)
    rc = lib.trial_hash_noalloc(
        _ptr(packed), ctypes.c_void_p(off.ctypes.data), off.size - 1, l, k, s, seed, t0, T, None,
        None, None, cap_c, cap_m, _ptr(out["cand_trial"]), _ptr(out["cand_key"]),
        _ptr(out["cand_cnt"]), _ptr(out["cand_off"]), _ptr(out["members"]), _ptr(tot),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out, tot.cpu().tolist()


def _same(P, packed, off, l, k, s, seed, t0, T, lib):
    ref = P.trial_hash(packed, off, l, k, s, seed, t0, T)
    C, M = ref["n_candidates"], ref["n_members"]
    rc, got, tot = _noalloc(lib, packed, off, l, k, s, seed, t0, T, C + 3, M + 5)
    assert rc == 0, lib.projection_last_error()
    assert tot == [C, M]
    for key in ("cand_trial", "cand_key", "cand_cnt", "members"):
        n = M if key == "members" else C
        assert torch.equal(got[key][:n], ref[key]), key
    assert torch.equal(got["cand_off"][:C + 1], ref["cand_off"])
    return C, M


def test_noalloc_matches_trial_hash_on_consecutive_calls(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    results = []
    for cfg, seed, T in ((1, 1001, 100), (3, 1003, 40), (1, 77, 60)):
        inst = instance_for_config(cfg)
        a = torch.from_numpy(inst.ascii).cuda()
        packed = P.projection_pack(a)
        prm = inst.params
        results.append(_same(P, packed, inst.seq_off, inst.l, prm["k"], prm["s"], seed, 0, T,
                             native_lib))
    assert all(C > 0 and M > 0 for C, M in results)


def test_noalloc_worked_example_bucket(native_lib, fig1):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    packed = P.projection_pack(torch.frombuffer(bytearray("".join(fig1).encode()),
                                                dtype=torch.uint8).cuda())
    off = np.arange(8, dtype=np.int64) * 40
    h = P.trial_hash_noalloc(packed, off, 8, 5, 4, 0, 0, 1, 16, 64,
                             positions_in=np.array([0, 1, 2, 5, 6], np.int32))
    assert h["cand_key"].cpu().tolist() == [177, 726] and h["cand_cnt"].cpu().tolist() == [7, 5]


def test_noalloc_refuses_work_beyond_its_scratch(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    inst = instance_for_config(1)
    packed = P.projection_pack(torch.from_numpy(inst.ascii).cuda())
    cap_m = (8 << 20) // 8 + 1  # the compaction list alone exceeds the array
    big = torch.zeros(1, dtype=torch.int32, device="cuda")
    off = np.ascontiguousarray(inst.seq_off)
    tot = torch.full((2,), -9, dtype=torch.int64, device="cuda")
    co = torch.zeros(2, dtype=torch.int64, device="cuda")
    rc = native_lib.trial_hash_noalloc(
        _ptr(packed), ctypes.c_void_p(off.ctypes.data), inst.t, 11, 7, 4, 1, 0, 10, None, None,
        None, 1, cap_m, _ptr(big), _ptr(big), _ptr(big), _ptr(co), _ptr(big), _ptr(tot),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -3 and b"scratch" in native_lib.projection_last_error()
    assert tot.cpu().tolist() == [-9, -9]  # nothing was launched


def _random_input(seed, t, nmin, nmax):
    rng = np.random.default_rng(seed)
    lens = rng.integers(nmin, nmax + 1, t)
    seqs = [np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, n)].tobytes() for n in lens]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return b"".join(seqs), off


def _parts(k, x):
    """Key-range parts per trial, as the header states them."""
    nb = 4 ** k
    if nb <= 32768:
        return 1
    if x <= 65535:
        return max(1, nb // 65536)
    return nb // 32768


def test_noalloc_many_parts_over_a_large_input(native_lib):
    """k = 9 over x > 65,535 l-mers: 8 key-range parts of u32 counters, each
    CTA scanning every l-mer of its trial (trial_hash partitions the pairs
    first instead).  Bit for bit the same lists."""
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    ascii, off = _random_input(8, 6, 19000, 21000)
    l, k, s = 16, 9, 2
    x = int(np.sum(np.diff(off) - l + 1))
    assert x > 65535 and _parts(k, x) == 8
    packed = P.projection_pack(torch.frombuffer(bytearray(ascii), dtype=torch.uint8).cuda())
    for seed, T in ((5, 6), (6, 3)):
        C, M = _same(P, packed, off, l, k, s, seed, 1, T, native_lib)
        assert C > 0 and M > 0


def _need(t, n_trials, parts, cap_m):
    a = lambda v: (v + 255) // 256 * 256  # noqa: E731
    return a(8 * (t + 1)) + a(8 * n_trials * parts) + a(16 * n_trials * parts) + a(8 * cap_m)


def test_noalloc_scratch_formula_is_exact(native_lib):
    """The largest trial count the header's scratch formula allows is accepted;
    one more is refused with ECAPACITY before anything is launched.  Three
    counter layouts: one part (k = 7), u16 parts (k = 9, x <= 65,535), u32 parts
    (k = 9, x > 65,535)."""
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    limit = 8 << 20
    inst = instance_for_config(1)
    big_ascii, big_off = _random_input(8, 6, 19000, 21000)
    shapes = [(inst.ascii.tobytes(), inst.seq_off, 11, 7, 4),
              (inst.ascii.tobytes(), inst.seq_off, 11, 9, 3),
              (big_ascii, big_off, 16, 9, 3)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for ascii, off, l, k, s in shapes:
        t = off.size - 1
        x = int(np.sum(np.diff(off) - l + 1))
        parts = _parts(k, x)
        # leave room for about 150 trials next to the compaction list
        cap_m = (limit - 256 - 24 * parts * 150) // 8
        n_max = 0
        while _need(t, n_max + 1, parts, cap_m) <= limit:
            n_max += 1
        assert 100 <= n_max <= 200
        packed = P.projection_pack(torch.frombuffer(bytearray(ascii), dtype=torch.uint8).cuda())
        offc = np.ascontiguousarray(off, np.int64)
        buf_c = torch.zeros(16, dtype=torch.int32, device="cuda")
        buf_o = torch.zeros(17, dtype=torch.int64, device="cuda")
        buf_m = torch.zeros(cap_m, dtype=torch.int32, device="cuda")
        for n, want_rc in ((n_max, 0), (n_max + 1, -3)):
            tot = torch.full((2,), -9, dtype=torch.int64, device="cuda")
            rc = native_lib.trial_hash_noalloc(
                _ptr(packed), ctypes.c_void_p(offc.ctypes.data), t, l, k, s, 3, 0, n, None, None,
                None, 16, cap_m, _ptr(buf_c), _ptr(buf_c), _ptr(buf_c), _ptr(buf_o), _ptr(buf_m),
                _ptr(tot), stream)
            assert rc == want_rc, (k, x, n, native_lib.projection_last_error())
            if want_rc == 0:
                C, M = tot.cpu().tolist()
                ref = P.trial_hash(packed, off, l, k, s, 3, 0, n)
                assert (C, M) == (ref["n_candidates"], ref["n_members"])
            else:
                assert tot.cpu().tolist() == [-9, -9]
