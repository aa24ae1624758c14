"""CPU checks of the C ABI: the library loads, exports every function that
include/projection.h declares, and its host-side parameter choice agrees with
the oracle.  No device work is launched."""
import ctypes
import os
import re

import pytest

import oracle as O
from tests.conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "projection.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^(?:const\s+)?(?:int|int64_t|void|char)\s*\*?\s*(\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("projection_find", "trial_hash", "em_refine", "projection_result_free"):
        assert n in names


def test_library_exports_every_declared_symbol(native_lib):
    from paper_1605_06904_gb300 import _native
    for n in _declared():
        assert hasattr(native_lib, n), n
    assert set(_native.SIGNATURES) == set(_declared())
    # the binding's names are the C names
    import paper_1605_06904_gb300 as P
    for n in _declared():
        if n not in ("projection_last_error", "projection_result_free"):
            assert hasattr(P, n), n


def test_library_targets_sm_103a_only():
    from paper_1605_06904_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("lens,l,d,k,s,m", [
    ([600] * 20, 11, 2, 0, 0, 0), ([600] * 20, 15, 4, 7, 4, 0), ([1000] * 20, 18, 6, 8, 3, 0),
    ([300, 900, 1200, 450] * 5, 13, 3, 8, 4, 0), ([5000] * 20, 8, 2, 4, 0, 7)])
def test_default_params_match_oracle(native_lib, lens, l, d, k, s, m):
    import paper_1605_06904_gb300 as P
    assert P.projection_default_params(lens, l, d, k, s, m) == O.default_params(lens, l, d, k, s, m)


def test_default_params_rejects_k_above_l_minus_d(native_lib):
    import paper_1605_06904_gb300 as P
    with pytest.raises(P.ProjectionError) as e:
        P.projection_default_params([600] * 20, 11, 2, k=10)
    assert e.value.status == -1


def test_packed_words(native_lib):
    import paper_1605_06904_gb300 as P
    assert [P.projection_packed_words(n) for n in (0, 1, 16, 17, 1000)] == [0, 1, 1, 2, 63]


def test_last_error_is_empty_after_success(native_lib):
    native_lib.projection_packed_words(3)
    import paper_1605_06904_gb300 as P
    P.projection_default_params([50] * 3, 10, 2)
    assert native_lib.projection_last_error() == b""
