"""Host-side helpers of the sweeps, the experiments and the surrogate (no
GPU): the parameter draws, the equilibrium rule for Laplace fits (R12b), the
interface width and deformation measures against closed forms, and the
surrogate's target transform."""
import math

import numpy as np
import pytest

import lbm_inputs as I
import paper_1412_7228_gb300 as P
from paper_1412_7228_gb300 import experiments as E
from paper_1412_7228_gb300 import sweep as SW
from paper_1412_7228_gb300 import surrogate as SU


def test_sweep_draws_are_seeded_and_in_range():
    """64 droplets, L uniform over {128, 256, 512, 1024}, R0 = 0.2 L,
    T/Tc in [0.6, 0.85], kappa in [0, 0.6], A in [-0.2, -0.1] shifted by
    -0.7 (reading R-A)."""
    a = SW.sweep_droplets(64, 7228)
    b = SW.sweep_droplets(64, 7228)
    assert [(d.L, d.radius, d.t_over_tc, d.A, d.kappa) for d in a] == \
        [(d.L, d.radius, d.t_over_tc, d.A, d.kappa) for d in b]
    assert {d.L for d in a} == {128, 256, 512, 1024}
    for d in a:
        assert d.radius == 0.2 * d.L
        assert 0.6 <= d.t_over_tc <= 0.85 and 0.0 <= d.kappa <= 0.6 and -0.9 <= d.A <= -0.8
    X = SU.sample_params(500, seed=1)
    assert X.shape == (500, 3) and np.array_equal(X, SU.sample_params(500, seed=1))
    assert not np.array_equal(X, SU.sample_params(500, seed=2))
    assert X[:, 0].min() >= 0.6 and X[:, 0].max() <= 0.85
    assert X[:, 1].min() >= -0.9 and X[:, 1].max() <= -0.8
    assert X[:, 2].min() >= 0.0 and X[:, 2].max() <= 0.6


def test_surrogate_targets_round_trip():
    """The network learns log sigma and log u_max, the densities as they are."""
    rng = np.random.default_rng(3)
    Y = np.column_stack([rng.uniform(1e-3, 2e-2, 50), rng.uniform(0.3, 0.4, 50), rng.uniform(0.005, 0.02, 50),
                         rng.uniform(1e-4, 1e-2, 50)])
    Z = SU.to_net(Y)
    assert np.array_equal(Z[:, 1:3], Y[:, 1:3])
    assert np.allclose(Z[:, 0], np.log(Y[:, 0]), rtol=0, atol=0) and np.allclose(Z[:, 3], np.log(Y[:, 3]))
    assert np.allclose(SU.from_net(Z), Y, rtol=1e-14, atol=0)


def _settled(**kw):
    _, rg, rl = SW.cs_eos(0.7)
    d = SW.Droplet(256, 40.0, 0.7, -0.85, 0.0)
    d.dp, d.R_eq, d.rho_l, d.rho_g, d.status, d.n_samples, d.R_drift = 1e-3, 38.0, rl, rg, 0, 101, 1e-5
    for k, v in kw.items():
        setattr(d, k, v)
    return d, rg, rl


def test_equilibrium_rule_for_laplace_fits():
    """R12b: a drop enters a fit when it is stable, still a liquid drop (its
    core denser than the gas by half the Maxwell gap) and its equimolar
    radius moved by less than 1e-3 over the sampling window."""
    d, rg, rl = _settled()
    assert SW.in_equilibrium(d)
    assert not SW.in_equilibrium(_settled(status=P.lbm.LBM_EUNSTABLE)[0])
    assert not SW.in_equilibrium(_settled(dp=float("nan"))[0])
    assert not SW.in_equilibrium(_settled(R_eq=0.0)[0])
    assert not SW.in_equilibrium(_settled(rho_l=rg + 0.4 * (rl - rg))[0])       # evaporated: gas inside
    assert SW.in_equilibrium(_settled(rho_l=rg + 0.6 * (rl - rg))[0])
    assert not SW.in_equilibrium(_settled(R_drift=-2e-3)[0])                    # still shrinking
    assert SW.in_equilibrium(_settled(R_drift=-2e-3, n_samples=1)[0])           # one sample: no drift known


def test_interface_width_of_a_tanh_profile():
    """The 10-90 % width of rho_g + (rho_l - rho_g)/2 (1 + tanh(2 x / W)) is
    W artanh(0.8); interpolating linearly between nodes widens an interface
    only a few nodes wide (3 % at W = 4, the Peng-Robinson interface's
    scale), and the error vanishes as W grows."""
    err = {}
    for W in (4.0, 16.0, 32.0):
        prof = I.slab_density(1024, 1, 7.0, 0.02, width=W)[0]
        err[W] = E.interface_width(prof) / (W * math.atanh(0.8)) - 1
    assert 0 < err[4.0] < 0.04 and abs(err[16.0]) < 0.005 and abs(err[32.0]) < 0.002


def test_deformation_of_circles_and_ellipses():
    """sum (rho - rho_g)(dx^2 - dy^2) / sum (rho - rho_g): zero for a circle,
    (a^2 - b^2)/4 for a uniform ellipse of semi-axes a (x) and b (y)."""
    rg = 0.02
    circle = I.droplet_density(256, 256, 35.0, 7.0, rg, width=0.5)
    assert abs(E.deformation(circle, rg)) < 1e-9 * 35.0 ** 2
    ell = I.ellipse_density(256, 256, 40.0, 30.0, 7.0, rg, width=0.5)
    assert abs(E.deformation(ell, rg) / ((40.0 ** 2 - 30.0 ** 2) / 4) - 1) < 0.02
    tall = np.ascontiguousarray(ell.T)
    assert E.deformation(tall, rg) == pytest.approx(-E.deformation(ell, rg), rel=1e-12)
