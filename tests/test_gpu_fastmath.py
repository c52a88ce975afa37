"""The FP64 step's reciprocal, division and square root (Newton-Raphson and
Goldschmidt steps from the hardware estimates) against the IEEE-rounded
results CUDA computes, on the device: within 1 ulp over the arguments the
step meets (densities, EOS denominators and psi radicands of the workloads
span about 1e-4 to 16), and the square root's signed zeros and NaN."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_7228_gb300 as P
    return P


@pytest.mark.parametrize("lo,hi", [(1e-8, 1e-4), (1e-4, 1.0), (1e-3, 0.6), (1.0, 16.0), (16.0, 1e6)])
def test_within_one_ulp_of_ieee(P, lo, hi):
    r = P.lbm_fp64_math_check(lo, hi, 1 << 24)
    assert r["rcp_ulp"] <= 1 and r["div_ulp"] <= 1 and r["sqrt_ulp"] <= 1, r
    assert r["sqrt_special_ok"], r


def test_arguments_are_checked(P):
    for lo, hi, n in ((0.0, 1.0, 10), (1.0, 0.5, 10), (1.0, float("inf"), 10), (1.0, 2.0, 0),
                      (float("nan"), 2.0, 10)):
        with pytest.raises(P.LbmError) as ei:
            P.lbm_fp64_math_check(lo, hi, n)
        assert ei.value.code == P.lbm.LBM_EINVAL
