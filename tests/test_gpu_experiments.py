"""The paper's experiments on the GPU path, against the numbers and
relations it prints (Sections 3.1, 4.1, 4.2) and the oracle's Eq. 17."""
import warnings

import numpy as np
import pytest

import lbm_inputs as I
import oracle as O
from oracle import analysis as An

warnings.filterwarnings("ignore", category=Warning, module="scipy")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_7228_gb300 import experiments
    return experiments


@pytest.fixture(scope="module")
def method1(E):
    return E.method1(As=(-0.9, -0.5, 0.0, 0.5, 0.99), steps_drop=6000, steps_slab=20000)


def test_fig2_flat_densities_follow_eq17_and_gas_moves_25_percent(method1):
    """Section 3.1.2: both coexistence densities move with A and the gas
    density changes by about 25 % from A = 1 to -0.9; each slab sits on the
    mechanical-stability coexistence of Eq. 17."""
    v = O.Params(eos=O.EOS_VDW, a=9 / 49, b=2 / 21, R=1.0, K=0.3)
    _, Tc, _ = An.critical_point(v)
    v.T = 0.9 * Tc
    for A, rl, rg in zip(method1["A"], method1["rho_l"], method1["rho_g"]):
        v.A = A
        eg, el, _ = An.mechanical_stability(v)
        assert abs(rl / el - 1) < 2e-4 and abs(rg / eg - 1) < 2e-3, A
    change = method1["rho_g"][0] / method1["rho_g"][-1] - 1
    assert 0.22 < change < 0.28


def test_fig1_sigma_falls_almost_linearly_with_A(method1):
    A = np.array(method1["A"][:-1])
    s = np.array(method1["sigma"][:-1])
    assert np.all(np.diff(s) < 0)
    c = np.polyfit(A, s, 1)
    r2 = 1 - ((s - np.polyval(c, A)) ** 2).sum() / ((s - s.mean()) ** 2).sum()
    assert r2 > 0.99
    assert abs(method1["sigma"][1] / 0.0459 - 1) < 0.05          # A = -0.5, the value quoted from Fig. 3


def test_peng_robinson_interface_ratio_width_and_sigma(E):
    """Section 4.1: density ratio 430 (the calibration of a), interface about
    4 nodes wide, and sigma(kappa = 0) = 0.16 as Section 4.2 uses it."""
    eos = E.pr_eos()
    b_rl, b_rg = E.pr_coexistence()
    assert abs(b_rl / b_rg / 430 - 1) < 0.02
    b = __import__("paper_1412_7228_gb300").lbm.Batch([128], [4], 2)
    b.set_params(0, eos, -0.3, 0.0, G=-1.0, s=E.S_ONES, rho_ref=0.0167)
    b.init_density(0, I.slab_density(128, 4, 7.17, 0.0167, width=4.0))
    b.step(30000)
    w = E.interface_width(b.read_fields(0, which=("rho",))["rho"].mean(axis=0))
    b.close()
    assert 3.0 < w < 5.0
    pl = E.pr_laplace(kappas=(0.0, 0.9), steps=20000)
    f0, f9 = pl["fits"][0.0], pl["fits"][0.9]
    assert f0["r2"] > 0.999 and f9["r2"] > 0.999
    assert abs(f0["sigma"] / 0.16 - 1) < 0.05
    assert abs(f9["sigma"] / f0["sigma"] / 0.1 - 1) < 0.10


def test_cylinder_oscillation_period_against_eq30(E):
    """Section 4.2: an elliptic cylinder oscillates with the period of Eq. 30
    (2 pi outside the root) within 10 %; the paper reports 3.5-16 %."""
    pl = E.pr_laplace(kappas=(-1.0, 0.0), steps=20000)
    for k in (-1.0, 0.0):
        o = E.oscillation(k, 0.05, sigma=pl["fits"][k]["sigma"], steps=12000 if k < 0 else 16000)
        assert abs(o["rel_err"]) < 0.10, (k, o["period"], o["theory"])
