"""Failure detection without a GPU fault: a kernel waits on a barrier that
nothing arrives on, gives up after a short limit, and reports PROJ_ETIMEOUT;
the CUDA context stays usable for the next search."""
import time

import numpy as np
import pytest
import torch

from synth import planted_instance

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    rc = P.projection_selftest_wait(50_000_000)  # 50 ms
    dt = time.perf_counter() - t0
    assert rc == -5, native_lib.projection_last_error()
    assert dt < 5.0
    assert b"expired" in native_lib.projection_last_error()
    # the context is still usable
    inst = planted_instance(3, 0, 8, 120, 9, 1)
    r = P.projection_find(inst.ascii, inst.seq_off, 9, 1, 5, 3, 6, seed=1, em_iters=2,
                          precision=P.PROJ_EM_BF16_SPLIT)
    assert r["status"] == 0 and len(r["consensus"]) == 9
    assert torch.cuda.synchronize() is None


def test_selftest_rejects_bad_limits(native_lib):
    import paper_1605_06904_gb300 as P
    assert P.projection_selftest_wait(0) == -1
    assert P.projection_selftest_wait(10**10) == -1


def test_trial_hash_rejects_bad_arguments_without_launching(native_lib):
    import paper_1605_06904_gb300 as P
    packed = P.projection_pack(torch.frombuffer(bytearray(b"ACGT" * 40), dtype=torch.uint8).cuda())
    with pytest.raises(P.ProjectionError) as e:
        P.trial_hash(packed, np.array([0, 160]), 8, 11, 3, 0, 0, 2)  # k > 10
    assert e.value.status == -1
    with pytest.raises(P.ProjectionError):
        P.trial_hash(packed, np.array([0, 5, 160]), 8, 5, 3, 0, 0, 2)  # sequence shorter than l
