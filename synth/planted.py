"""Planted (l,d)-motif instances (Section 2's (l,d) variant; Section 5's challenge
problems of t = 20 sequences of 600-1000 bp).

Recipe (stated here because both sides of every comparison read it):
  * background: iid uniform over A/C/G/T, or a first-order Markov chain with 40%
    GC content (stationary P(A)=P(T)=0.3, P(C)=P(G)=0.2; transition
    T[a][b] = 0.8*pi[b] + 0.2*[a == b], whose stationary law is pi);
  * motif: a uniform random l-mer;
  * each occurrence: exactly d distinct positions of the motif replaced by one
    of the three other bases (uniform), written at a uniform start in [0, n-l];
  * OOPS: every sequence holds one occurrence; ZOOPS: a random subset of the
    sequences (a fraction `zoops_frac`) does.

All randomness comes from numpy's PCG64 raw 64-bit output (a stream that is
stable across numpy versions), seeded by (seed, instance) through SeedSequence,
and mapped to integers with explicit multiply-shift arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LETTERS = np.frombuffer(b"ACGT", dtype=np.uint8)


class _Stream:
    def __init__(self, seed: int, instance: int):
        self._bg = np.random.PCG64(np.random.SeedSequence([int(seed), int(instance)]))

    def raw(self, n: int) -> np.ndarray:
        return self._bg.random_raw(n).astype(np.uint64)

    def below(self, m: int, n: int | None = None):
        """Uniform integer(s) in [0, m) from the top 32 bits (m < 2^32)."""
        r = (self.raw(1 if n is None else n) >> np.uint64(32)) * np.uint64(m) >> np.uint64(32)
        return int(r[0]) if n is None else r.astype(np.int64)

    def uniform(self, n: int) -> np.ndarray:
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Instance:
    """One motif-finding input: t ASCII sequences and what was planted in it."""
    seqs: list            # list[bytes]
    l: int
    d: int
    motif: str
    starts: np.ndarray    # int64[t], -1 where nothing was planted
    params: dict = field(default_factory=dict)

    @property
    def t(self) -> int:
        return len(self.seqs)

    @property
    def lens(self) -> np.ndarray:
        return np.array([len(q) for q in self.seqs], np.int64)

    @property
    def seq_off(self) -> np.ndarray:
        off = np.zeros(self.t + 1, np.int64)
        off[1:] = np.cumsum(self.lens)
        return off

    @property
    def ascii(self) -> np.ndarray:
        return np.frombuffer(b"".join(self.seqs), dtype=np.uint8).copy()

    @property
    def n_lmers(self) -> int:
        return int(np.maximum(self.lens - self.l + 1, 0).sum())


def _background(st: _Stream, n: int, kind: str) -> np.ndarray:
    if kind == "uniform":
        return LETTERS[st.below(4, n)]
    if kind == "markov_gc40":
        # order of LETTERS: A C G T
        pi = np.array([0.3, 0.2, 0.2, 0.3])
        T = 0.8 * pi[None, :] + 0.2 * np.eye(4)
        cdf = np.cumsum(T, axis=1)
        u = st.uniform(n)
        out = np.empty(n, np.int64)
        a = int(np.searchsorted(np.cumsum(pi), u[0], side="right"))
        out[0] = min(a, 3)
        for i in range(1, n):
            a = int(np.searchsorted(cdf[a], u[i], side="right"))
            a = min(a, 3)
            out[i] = a
        return LETTERS[out]
    raise ValueError(kind)


def planted_instance(seed: int, instance: int, t: int, n, l: int, d: int,
                     background: str = "uniform", zoops_frac: float = 1.0) -> Instance:
    """t sequences of length n (an int, or a list of t ints) with a planted (l,d) motif."""
    st = _Stream(seed, instance)
    lens = [int(n)] * t if np.isscalar(n) else [int(v) for v in n]
    motif = LETTERS[st.below(4, l)].copy()
    if zoops_frac >= 1.0:
        has = np.ones(t, bool)
    else:
        nplant = int(round(zoops_frac * t))
        order = np.argsort(st.raw(t), kind="stable")
        has = np.zeros(t, bool)
        has[order[:nplant]] = True
    seqs, starts = [], np.full(t, -1, np.int64)
    for i in range(t):
        s = _background(st, lens[i], background)
        if has[i] and lens[i] >= l:
            occ = motif.copy()
            # d distinct positions: partial Fisher-Yates on 0..l-1
            perm = np.arange(l)
            for q in range(d):
                j = q + st.below(l - q)
                perm[q], perm[j] = perm[j], perm[q]
            for p in perm[:d]:
                others = LETTERS[LETTERS != occ[p]]
                occ[p] = others[st.below(3)]
            a = st.below(lens[i] - l + 1)
            s[a:a + l] = occ
            starts[i] = a
        seqs.append(s.tobytes())
    return Instance(seqs=seqs, l=l, d=d, motif=motif.tobytes().decode(), starts=starts)


AA_LETTERS = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", dtype=np.uint8)


def planted_protein(seed: int, instance: int, t: int, n, l: int, d: int) -> Instance:
    """Protein counterpart of planted_instance: iid uniform residues over the 20
    amino-acid letters, a uniform random motif, and in every sequence one
    occurrence with exactly d distinct positions replaced by one of the 19
    other letters (uniform), at a uniform start."""
    st = _Stream(seed, instance)
    lens = [int(n)] * t if np.isscalar(n) else [int(v) for v in n]
    motif = AA_LETTERS[st.below(20, l)].copy()
    seqs, starts = [], np.full(t, -1, np.int64)
    for i in range(t):
        s = AA_LETTERS[st.below(20, lens[i])]
        if lens[i] >= l:
            occ = motif.copy()
            perm = np.arange(l)
            for q in range(d):
                j = q + st.below(l - q)
                perm[q], perm[j] = perm[j], perm[q]
            for p in perm[:d]:
                others = AA_LETTERS[AA_LETTERS != occ[p]]
                occ[p] = others[st.below(19)]
            a = st.below(lens[i] - l + 1)
            s[a:a + l] = occ
            starts[i] = a
        seqs.append(s.tobytes())
    return Instance(seqs=seqs, l=l, d=d, motif=motif.tobytes().decode(), starts=starts)


# The five workloads: sizes and parameters of the planted challenge problems.
CONFIGS = {
    1: dict(name="planted(11,2) t=20 n=600", t=20, n=600, l=11, d=2, k=7, s=4, m=100,
            em_iters=5, beta=0.25),
    2: dict(name="planted(15,4) t=20 n=600", t=20, n=600, l=15, d=4, k=7, s=4, m=0,
            em_iters=5, beta=0.25),
    3: dict(name="planted(18,6) t=20 n=1000", t=20, n=1000, l=18, d=6, k=8, s=3, m=2000,
            em_iters=8, beta=0.25),
    5: dict(name="markov-gc40 zoops(20,5) t=2000 n=500", t=2000, n=500, l=20, d=5, k=10, s=4,
            m=500, em_iters=10, beta=0.25, background="markov_gc40", zoops_frac=0.6,
            top=1024),
}


def instance_for_config(cfg: int, instance: int = 0) -> Instance:
    c = CONFIGS[cfg]
    inst = planted_instance(1000 + cfg, instance, c["t"], c["n"], c["l"], c["d"],
                            background=c.get("background", "uniform"),
                            zoops_frac=c.get("zoops_frac", 1.0))
    inst.params = {k: v for k, v in c.items() if k in ("k", "s", "m", "em_iters", "beta", "top")}
    return inst


MIX_LD = [(11, 2), (13, 3), (15, 4), (17, 5), (19, 6)]


def mix_instances(count: int = 256, seed: int = 1004) -> list:
    """Serving-shaped mix: t ~ U[10,40], n ~ U[300,1200], (l,d) from MIX_LD,
    k = min(l-d, ceil(log4(t*n))), s = 4 (m is left to the Section 5 bound)."""
    st = _Stream(seed, 10**6)
    out = []
    for q in range(count):
        t = 10 + st.below(31)
        n = 300 + st.below(901)
        l, d = MIX_LD[st.below(len(MIX_LD))]
        k = min(l - d, math.ceil(math.log(t * n, 4)))
        inst = planted_instance(seed, q, t, n, l, d)
        inst.params = dict(k=k, s=4, m=0, em_iters=5, beta=0.25)
        out.append(inst)
    return out
