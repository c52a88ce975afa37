"""Batched droplet sweeps on the GPU: Laplace-law fits against the oracle,
and the batched launch against one-by-one runs."""
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
def SW():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_7228_gb300 import sweep
    return sweep


def oracle_laplace(kappa, radii, N, steps, tr=0.7, A=-0.85, gap=10.0):
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A, kappa=kappa, s=list(S_CFG))
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, tr * Tc)
    rg, rl, _ = An.maxwell(p)
    dps, Rs = [], []
    for R in radii:
        f = O.init_equilibrium(I.droplet_density(N, N, R, rl, rg))
        O.step(p, f, steps)
        d = An.pressure_jump(p, O.macro(p, f)[0], N / 2, N / 2, R / 2, R + gap)
        dps.append(d["dp"])
        Rs.append(d["R_eq"])
    return An.laplace_fit(dps, Rs)


def test_laplace_sweep_matches_oracle_and_kappa_law(SW):
    """sigma from the batched FP32 sweep within 1e-3 of the FP64 oracle's,
    r^2 >= 0.999, and sigma(0.5)/sigma(0) within 8 % of 1 - kappa: Eq. 28 is
    the leading order of a Taylor expansion, and this Carnahan-Starling
    interface (2-3 nodes wide) is sharper than the paper's K = 0.3 van der
    Waals one, where the oracle lands within 3 % (measured here: 5.4 %)."""
    radii = (10, 14, 18)
    fits, info = SW.laplace_sweep(radii=radii, kappas=(0.0, 0.3, 0.5), t_over_tc=(0.7,), L_=64, steps=4000,
                                  autotune=False)
    by_k = {f.kappa: f for f in fits}
    assert set(by_k) == {0.0, 0.3, 0.5}
    assert all(f.r2 >= 0.999 for f in fits)
    sig_o, _, r2_o = oracle_laplace(0.3, radii, 64, 4000)
    assert abs(by_k[0.3].sigma / sig_o - 1) <= 1e-3
    assert abs(by_k[0.5].sigma / by_k[0.0].sigma / 0.5 - 1) <= 0.08


def test_batched_equals_sequential(SW):
    drops = [SW.Droplet(L, 0.25 * L, tr, -0.85, k) for L, tr, k in
             ((64, 0.7, 0.1), (96, 0.75, 0.4), (128, 0.65, 0.0), (48, 0.8, 0.6))]
    seq = [SW.Droplet(d.L, d.radius, d.t_over_tc, d.A, d.kappa) for d in drops]
    SW.run_batch(drops, 300, autotune=True)
    SW.run_sequential(seq, 300)
    for a, b in zip(drops, seq):
        assert a.status == 0 and b.status == 0
        assert a.dp == b.dp and a.R_eq == b.R_eq and a.umax == b.umax
