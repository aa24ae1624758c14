"""The measurement helper behind the bucket kernels' roofline: the
shared-memory histogram rate must be a plausible positive rate for every k the
bucket kernels support, and no slower for small histograms than for large
ones by more than the expected bank-conflict spread."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(native_lib):
    import paper_1605_06904_gb300 as P
    torch.cuda.set_device(0)
    return P


@pytest.mark.parametrize("k", [4, 7, 8, 10])
def test_hist_peak_is_plausible(P, k):
    r = P.projection_hist_peak(k)
    # 152 SMs x ~2 GHz: at least one increment per SM every 100 clocks, at most
    # 128 per clock per SM
    assert 3e9 < r < 4e13, r


def test_hist_peak_rejects_bad_k(P):
    with pytest.raises(P.ProjectionError):
        P.projection_hist_peak(11)
