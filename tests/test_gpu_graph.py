"""CUDA-graph replay and the EM schedule autotuner.

The EM iterations (and, for batches, the finalisation) run as a captured graph
whose executable form is updated in place between calls.  With the schedule
pinned (PROJ_AUTOTUNE=0) the replay must give bit-identical results to the
same launches issued directly (PROJ_GRAPHS=0); reusing the executable graph
across calls of different shapes must not leak one call's parameters into the
next; and every schedule the autotuner may pick must agree with the oracle."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np
import torch
import paper_1605_06904_gb300 as P
from synth import planted_instance
torch.cuda.set_device(0)
out = {}
inst = planted_instance(1001, 0, 20, 600, 11, 2)
r = P.projection_find(inst.ascii, inst.seq_off, 11, 2, 7, 4, 30, seed=5, em_iters=5,
                      pseudocount=0.25, precision=P.PROJ_EM_BF16_SPLIT)
out["single"] = [r["loglik"].hex(), r["consensus"], r["sites"].tolist(),
                 [float(v).hex() for v in r["pwm"].ravel()]]
insts = [planted_instance(700 + q, 0, t, n, l, d) for q, (t, n, l, d) in
         enumerate([(12, 400, 11, 2), (20, 600, 15, 4), (9, 900, 13, 3)])]
res = P.projection_find_batch([i.seqs for i in insts], [i.l for i in insts], [i.d for i in insts],
                              [7, 7, 7], [4, 4, 4], [20, 25, 15], [3, 4, 5], em_iters=5,
                              pseudocount=0.25)
out["batch"] = [[g["loglik"].hex(), g["consensus"], g["sites"].tolist()] for g in res]
print("JSON" + json.dumps(out))
"""


def _run_child(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    p = subprocess.run([sys.executable, "-c", _CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("JSON")][-1]
    return json.loads(line[4:])


def test_graph_replay_equals_direct_launches(native_lib):
    a = _run_child({"PROJ_GRAPHS": "1", "PROJ_AUTOTUNE": "0"})
    b = _run_child({"PROJ_GRAPHS": "0", "PROJ_AUTOTUNE": "0"})
    assert a == b


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


def test_graph_reuse_across_shapes(P):
    from synth import planted_instance
    # same shape with other data (graph updated in place), another kernel
    # variant (re-instantiated), then the first call again
    calls = [(20, 600, 11, 2, 7, 4, 30, 5), (20, 600, 11, 2, 7, 4, 30, 9),
             (14, 500, 15, 4, 7, 4, 40, 5), (20, 600, 11, 2, 7, 4, 30, 9),
             (20, 600, 11, 2, 7, 4, 30, 5)]
    got = []
    for t, n, l, d, k, s, m, seed in calls:
        inst = planted_instance(1001, 0, t, n, l, d)
        got.append(P.projection_find(inst.ascii, inst.seq_off, l, d, k, s, m, seed=seed,
                                     em_iters=5, pseudocount=0.25,
                                     precision=P.PROJ_EM_BF16_SPLIT))
    for i, j in ((0, 4), (1, 3)):
        a, c = got[i], got[j]
        assert a["n_candidates"] == c["n_candidates"]
        assert a["loglik"] == c["loglik"] and a["consensus"] == c["consensus"]
        assert np.array_equal(a["sites"], c["sites"]) and np.array_equal(a["pwm"], c["pwm"])
    assert got[0]["n_candidates"] != got[1]["n_candidates"]
    assert got[2]["l"] == 15 and len(got[2]["consensus"]) == 15


@pytest.mark.parametrize("sched", ["2,1", "2,2", "2,3", "2,4", "1,1", "1,4", "1,1,4", "1,2,4",
                                   "1,3,4"])
def test_every_em_schedule_matches_oracle(P, sched, monkeypatch):
    """Each schedule (CTAs per SM, rounds of CTA slots filled by the sequence
    groups, and the kernel's 64- or 128-l-mer tiles) splits the work differently; each must stay within the BF16-split
    tolerances of the FP64 oracle."""
    import oracle as O
    from synth import planted_instance
    from tests.conftest import ll_tol, oracle_theta0_sample
    monkeypatch.setenv("PROJ_EM_SCHED", sched)
    inst = planted_instance(1002, 0, 20, 600, 15, 4)
    codes = O.encode(inst.ascii)
    th0 = oracle_theta0_sample(inst, 7, 4, 11, 400, 8)
    want_th, want_ll = O.em(codes, inst.seq_off, 15, O.background(codes), th0.astype(np.float64),
                            5, 0.25, nthreads=16)
    packed = P.projection_pack(torch.from_numpy(np.frombuffer(bytes(inst.ascii), np.uint8).copy())
                               .cuda())
    bg = P.projection_background(packed, inst.seq_off[-1])
    th, ll = P.em_refine(packed, inst.seq_off, 15, bg, torch.from_numpy(th0).cuda(), 5, 0.25,
                         P.PROJ_EM_BF16_SPLIT)
    assert np.max(np.abs(th.cpu().numpy() - want_th)) <= 5e-5
    assert np.all(np.abs(ll.cpu().numpy() - want_ll) <= ll_tol(want_ll, inst.t, 1e-4))
