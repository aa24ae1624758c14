"""The measurement helpers behind the rooflines: the shared-memory histogram
rate must be a plausible positive rate for every k the bucket kernels support,
and the exp2 rate a plausible number of exponentials per clock and SM."""
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


def test_ex2_peak_is_plausible(P):
    r = P.projection_ex2_peak()
    # 152 SMs x ~2 GHz: between 1 and 128 exponentials per clock per SM
    assert 3e11 < r < 4e13, r
