"""Algorithm 2 step 1 on the device for a batch (Section 5): k, s and m of many
instances against the oracle's statement of the same formulas (host FP64).
m is an integer decided by FP64 arithmetic (a ceiling of a ratio of logs): both
sides use FP64, and the only tolerated difference is at a ratio within 1e-9 of
an integer, where the two libraries' last-place rounding may differ."""
import math

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


def _ratio(l, d, k, s, t, q=0.95):
    """log(1-q)/log B of the Section 5 bound (for the near-integer check)."""
    p = math.comb(l - d, k) / math.comb(l, k)
    B = sum(math.comb(t, c) * p ** c * (1 - p) ** (t - c) for c in range(0, min(s, t + 1)))
    return math.log(1 - q) / math.log(B) if 0 < B < 1 else None


def test_params_batch_matches_oracle(P):
    rng = np.random.default_rng(3)
    n = 400
    ld = [(11, 2), (13, 3), (15, 4), (17, 5), (19, 6), (20, 5), (9, 1), (8, 2)]
    pick = rng.integers(0, len(ld), n)
    l = np.array([ld[i][0] for i in pick], np.int32)
    d = np.array([ld[i][1] for i in pick], np.int32)
    t = rng.integers(5, 60, n).astype(np.int32)
    lens = rng.integers(200, 1500, n)
    x = (t.astype(np.int64) * (lens - l + 1)).astype(np.int64)
    # a third of the instances pass their own k (some giving no finite bound)
    kin = np.where(rng.random(n) < 0.33, rng.integers(4, 12, n), 0).astype(np.int32)
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(a).to(dev)
    k, s, m, st = P.projection_params_batch(T(t), T(x), T(l), T(d), k=T(kin))
    k, s, m, st = (v.cpu().numpy() for v in (k, s, m, st))
    for i in range(n):
        if kin[i] > l[i]:
            assert st[i] == -1
            continue
        ks = int(kin[i]) or int(l[i] - d[i] - 1)
        ss = max(3, math.ceil(2 * int(x[i]) / 4 ** ks))
        assert k[i] == ks and s[i] == ss
        want = O.m_bound(int(l[i]), int(d[i]), ks, ss, int(t[i]))
        if want < 0 or want > 1 << 24:
            assert st[i] == -2 and m[i] == 0
            continue
        assert st[i] == 0
        if m[i] != want:
            r = _ratio(int(l[i]), int(d[i]), ks, ss, int(t[i]))
            assert r is not None and abs(r - round(r)) < 1e-9 and abs(int(m[i]) - want) == 1


def test_params_batch_keeps_given_values_and_rejects_bad(P):
    dev = torch.device("cuda", 0)
    t = torch.tensor([20, 0, 20], dtype=torch.int32, device=dev)
    x = torch.tensor([11800, 100, 11800], dtype=torch.int64, device=dev)
    l = torch.tensor([11, 11, 11], dtype=torch.int32, device=dev)
    d = torch.tensor([2, 2, 11], dtype=torch.int32, device=dev)
    k, s, m, st = P.projection_params_batch(t, x, l, d, k=torch.tensor([7, 0, 0], dtype=torch.int32, device=dev),
                                            s=torch.tensor([4, 0, 0], dtype=torch.int32, device=dev),
                                            m=torch.tensor([100, 0, 0], dtype=torch.int32, device=dev))
    assert (int(k[0]), int(s[0]), int(m[0]), int(st[0])) == (7, 4, 100, 0)
    assert int(st[1]) == -1 and int(st[2]) == -1
