"""Coexistence densities of flat interfaces in FP32 deviation storage against
the FP64 oracle: the paper's Table 1 case (van der Waals, K = 0.3, 0.9 Tc,
A = -0.5, s = 1) and the Carnahan-Starling slab of the droplet workloads
(0.7 Tc, A = -0.85), each within 1e-3 relative after the same number of
steps, and the Table 1 densities the paper prints within 1e-3."""
import warnings

import numpy as np
import pytest

import lbm_inputs as I
import oracle as O
from oracle import analysis as An

warnings.filterwarnings("ignore", category=Warning, module="scipy")

pytestmark = pytest.mark.gpu
S_CFG = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]


@pytest.fixture(scope="module")
def X():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_7228_gb300 import experiments
    return experiments


def oracle_slab(op, rho0, steps):
    f = O.init_equilibrium(rho0)
    O.step(op, f, steps)
    return An.slab_densities(O.macro(op, f)[0])


def test_table1_flat_interface_in_fp32(X, golden):
    eos = X.vdw_eos(0.9, 0.3)
    rho0 = I.slab_density(128, 4, 5.8, 1.47, width=4.0)
    steps = 15000
    op = O.Params(eos=O.EOS_VDW, a=9 / 49, b=2 / 21, R=1.0, K=0.3, T=eos.T, A=-0.5, kappa=0.5, s=[1.0] * 9)
    rl_o, rg_o = oracle_slab(op, rho0, steps)
    (rl, rg), = X.slabs(eos, [(-0.5, 0.5)], 5.8, 1.47, steps=steps, precision=1)
    assert abs(rl / rl_o - 1) <= 1e-3 and abs(rg / rg_o - 1) <= 1e-3, (rl, rl_o, rg, rg_o)
    t1 = golden["table1_flat_interface"]
    assert abs(rl / t1["rho_l"] - 1) <= 1e-3 and abs(rg / t1["rho_g"] - 1) <= 1e-3


def test_carnahan_starling_slab_in_fp32(X):
    import paper_1412_7228_gb300 as P
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = 0.7 * Tc
    rg0, rl0, _ = P.lbm_eos_maxwell(eos)
    rho0 = I.slab_density(128, 4, rl0, rg0, width=4.0)
    steps = 20000
    op = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=eos.T, A=-0.85, kappa=0.3, s=S_CFG)
    rl_o, rg_o = oracle_slab(op, rho0, steps)
    (rl, rg), = X.slabs(eos, [(-0.85, 0.3)], rl0, rg0, steps=steps, s=S_CFG, precision=1)
    assert abs(rl / rl_o - 1) <= 1e-3 and abs(rg / rg_o - 1) <= 1e-3, (rl, rl_o, rg, rg_o)
