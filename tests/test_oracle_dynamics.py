"""Pins of the oracle's full time step against closed-form flows,
conservation laws, symmetries and Taylor limits (not against itself)."""
import math
import warnings

import numpy as np
import pytest

import lbm_inputs as I
import oracle as O
from oracle import analysis as An

warnings.filterwarnings("ignore", category=Warning, module="scipy")

S_CFG = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]


def cs_params(tr=0.7, A=-0.85, kappa=0.0, **kw):
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A, kappa=kappa, s=list(S_CFG), **kw)
    _, Tc, _ = An.critical_point(base)
    return An.with_T(base, tr * Tc)


@pytest.fixture(scope="module")
def droplet_state():
    p = cs_params(kappa=0.3)
    rg, rl, _ = An.maxwell(p)
    rho = I.droplet_density(48, 48, 12, rl, rg)
    return p, rho


def test_mass_is_conserved_to_round_off(droplet_state):
    p, rho = droplet_state
    f = O.init_equilibrium(rho)
    m0 = f.sum()
    O.step(p, f, 300)
    assert abs(f.sum() / m0 - 1) < 1e-13


def test_total_momentum_stays_zero_from_asymmetric_start():
    """sum_x F = 0 on a periodic lattice (Eq. 9 is antisymmetric in e), so the
    total momentum of a noisy state starting at rest stays at round-off."""
    p = cs_params(kappa=0.5)
    rho = I.spinodal_density(40, 36, rho0=0.25, amp=0.05, seed=11)
    f = O.init_equilibrium(rho)
    O.step(p, f, 150)
    ex, ey, _ = O.velocities()
    jx = (f * ex[:, None, None]).sum()
    jy = (f * ey[:, None, None]).sum()
    assert abs(jx) < 1e-12 * rho.size and abs(jy) < 1e-12 * rho.size


def test_uniform_body_force_adds_F_per_step():
    """With G = 0 and a constant force density, the total of j + F/2 grows by
    exactly N F per step (R2 and the (I - Lambda/2) S forcing)."""
    g = 1e-4
    p = O.Params(G=0.0, s=[1, 1.3, 0.7, 1, 1.2, 1, 1.2, 1.5, 1.5], fext_x=g, fext_y=-g / 2)
    f = O.init_equilibrium(np.full((8, 10), 0.7))
    O.step(p, f, 25)
    rho, ux, uy, *_ = O.macro(p, f)
    N = 80
    assert abs((rho * ux).sum() - N * g * 25.5) < 1e-13
    assert abs((rho * uy).sum() + N * g / 2 * 25.5) < 1e-13


@pytest.mark.parametrize("s_nu", [1.0, 1.6])
def test_poiseuille_matches_parabola(s_nu):
    """G = 0, half-way bounce-back walls, constant force density g: the
    steady profile is g/(2 rho nu) (y+1/2)(H-1/2-y) with nu = (1/s_nu - 1/2)/3.
    With s_q = 8(2 - s_nu)/(8 - s_nu) the wall sits exactly half-way."""
    H, g = 16, 1e-5
    s_q = 8 * (2 - s_nu) / (8 - s_nu)
    p = O.Params(G=0.0, s=[1, 1.1, 1.1, 1, s_q, 1, s_q, s_nu, s_nu], fext_x=g, walls_y=True)
    f = O.init_equilibrium(np.ones((H, 4)))
    O.step(p, f, 16000)
    rho, ux, uy, *_ = O.macro(p, f)
    nu = (1 / s_nu - 0.5) / 3
    y = np.arange(H)
    ua = g / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    assert np.abs(ux[:, 0] - ua).max() < 2e-6 * ua.max()
    assert np.abs(uy).max() < 1e-14


@pytest.mark.parametrize("s_nu", [1.0, 1.7])
def test_shear_wave_decays_with_lattice_viscosity(s_nu):
    L, U0 = 64, 1e-4
    y = np.arange(L)
    ux = np.broadcast_to((U0 * np.sin(2 * math.pi * y / L))[:, None], (L, 4)).copy()
    p = O.Params(G=0.0, s=[1, 1.1, 1.1, 1, 1.1, 1, 1.1, s_nu, s_nu])
    f = O.init_equilibrium(np.ones((L, 4)), ux, np.zeros_like(ux))
    O.step(p, f, 50)
    a1 = O.macro(p, f)[1][:, 0] @ np.sin(2 * math.pi * y / L)
    O.step(p, f, 400)
    a2 = O.macro(p, f)[1][:, 0] @ np.sin(2 * math.pi * y / L)
    k = 2 * math.pi / L
    nu_meas = -math.log(a2 / a1) / (k * k * 400)
    nu = (1 / s_nu - 0.5) / 3
    assert abs(nu_meas / nu - 1) < 2e-3


def test_streaming_direction_by_advection():
    """A transverse wave u_y = d sin(k x) on a uniform flow U moves to +x at
    speed U: its phase lags by k U t."""
    L, U, d = 64, 0.05, 1e-4
    x = np.arange(L)
    ux = np.full((4, L), U)
    uy = np.broadcast_to(d * np.sin(2 * math.pi * x / L)[None, :], (4, L)).copy()
    p = O.Params(G=0.0, s=[1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1.2, 1.2])
    f = O.init_equilibrium(np.ones((4, L)), ux, uy)
    k = 2 * math.pi / L

    def phase():
        v = O.macro(p, f)[2][0]
        return np.angle(np.fft.fft(v)[1])

    O.step(p, f, 20)
    ph1 = phase()
    O.step(p, f, 200)
    ph2 = phase()
    dphi = (ph2 - ph1 + math.pi) % (2 * math.pi) - math.pi
    assert abs(dphi / (-k * U * 200) - 1) < 0.02


def test_droplet_keeps_square_symmetry(droplet_state):
    p, rho = droplet_state
    f = O.init_equilibrium(rho)
    O.step(p, f, 200)
    r = O.macro(p, f)[0]
    scale = r.max()
    assert np.abs(r - r.T).max() < 1e-12 * scale
    mirror = np.roll(r[:, ::-1], 1, axis=1)          # x -> (nx - x) mod nx about the centre
    assert np.abs(r - mirror).max() < 1e-12 * scale


def test_kappa_zero_is_bitwise_the_unmodified_model(droplet_state):
    """kappa = 0 adds C = 0 and is bit-identical to never evaluating Q (R19)."""
    p, rho = droplet_state
    a = O.init_equilibrium(rho)
    b = a.copy()
    p0 = O.Params(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    p0.kappa = 0.0
    pn = O.Params(**{k: getattr(p0, k) for k in p0.__dataclass_fields__})
    pn.no_q = True
    O.step(p0, a, 120)
    O.step(pn, b, 120)
    assert a.tobytes() == b.tobytes()
    # and kappa != 0 does change the result
    c = O.init_equilibrium(rho)
    O.step(p, c, 120)
    assert np.abs(c - a).max() > 1e-8


def test_only_the_sign_of_G_matters(droplet_state):
    """psi scales as |G|^-1/2 so G psi^2 and every force are unchanged (R10)."""
    p, rho = droplet_state
    q = O.Params(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.G = -2.0
    a = O.init_equilibrium(rho)
    b = a.copy()
    O.step(p, a, 100)
    O.step(q, b, 100)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def _smooth_psi(L):
    k = 2 * math.pi / L
    x = np.arange(L)[None, :]
    y = np.arange(L)[:, None]
    psi = 1.0 + 0.2 * np.sin(k * x) * np.cos(k * y) + 0.1 * np.sin(k * y)
    px = 0.2 * k * np.cos(k * x) * np.cos(k * y)
    py = -0.2 * k * np.sin(k * x) * np.sin(k * y) + 0.1 * k * np.cos(k * y)
    pxx = -0.2 * k * k * np.sin(k * x) * np.cos(k * y)
    pyy = -0.2 * k * k * np.sin(k * x) * np.cos(k * y) - 0.1 * k * k * np.sin(k * y)
    pxy = -0.2 * k * k * np.cos(k * x) * np.sin(k * y)
    return psi, px, py, pxx, pyy, pxy


@pytest.mark.parametrize("A", [-0.5, 0.3])
def test_force_and_Q_taylor_limits(A):
    """Eq. 9 tends to -G psi grad psi and Eq. 23 (x G/2, R3) to Eq. 24, both
    with second-order error: doubling the wavelength cuts the error ~4x."""
    G, kappa = -1.0, 0.7
    p = O.Params(A=A, kappa=kappa, G=G)
    errs = []
    for L in (32, 64):
        psi, px, py, pxx, pyy, pxy = _smooth_psi(L)
        Fx, Fy, Qxx, Qyy, Qxy = O.force_q(p, psi)
        lap = pxx + pyy
        g2 = px * px + py * py
        iso = G / 12 * psi * lap + A * G / 12 * g2
        Qxx_t = kappa * (iso + G / 6 * psi * pxx + A * G / 6 * px * px)
        Qyy_t = kappa * (iso + G / 6 * psi * pyy + A * G / 6 * py * py)
        Qxy_t = kappa * (G / 6 * psi * pxy + A * G / 6 * px * py)
        eF = max(np.abs(Fx + G * psi * px).max(), np.abs(Fy + G * psi * py).max())
        eQ = max(np.abs(Qxx - Qxx_t).max(), np.abs(Qyy - Qyy_t).max(), np.abs(Qxy - Qxy_t).max())
        sF = np.abs(G * psi * px).max()
        sQ = np.abs(Qxx_t).max()
        errs.append((eF / sF, eQ / sQ))
    (f1, q1), (f2, q2) = errs
    assert 3.5 < f1 / f2 < 4.5 and f2 < 1e-2
    assert 3.5 < q1 / q2 < 4.5 and q2 < 1e-2


def test_small_A_diverges_for_cs_at_0p7():
    """The oracle reports instability for the CS droplet at 0.7 T_c with
    A = -0.152 within a few steps (Eq. 17 has no coexistence there)."""
    p = cs_params(A=-0.152)
    rg, rl, _ = An.maxwell(p)
    f = O.init_equilibrium(I.droplet_density(64, 64, 15, rl, rg))
    with pytest.raises(O.OracleUnstable):
        O.step(p, f, 50)


@pytest.mark.parametrize("rho0,nu_expect", [(1.0, 0.2), (3.0, 0.125), (6.0, 0.05), (0.5, 0.2)])
def test_density_dependent_viscosity_sets_the_shear_decay(rho0, nu_expect):
    """Section 4.2's density-dependent viscosity (linear in rho between the
    gas (1, 0.2) and liquid (5, 0.05) states, clamped): a shear wave in a
    uniform fluid of density rho0 decays with nu(rho0)."""
    L, U0 = 64, 1e-5
    y = np.arange(L)
    ux = np.broadcast_to((U0 * np.sin(2 * math.pi * y / L))[:, None], (L, 4)).copy()
    p = O.Params(G=0.0, s=[1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1.0, 1.0], var_visc=True, nu_g=0.2, nu_l=0.05,
                 visc_rho_g=1.0, visc_rho_l=5.0)
    f = O.init_equilibrium(np.full((L, 4), rho0), ux, np.zeros_like(ux))
    O.step(p, f, 50)
    a1 = O.macro(p, f)[1][:, 0] @ np.sin(2 * math.pi * y / L)
    O.step(p, f, 300)
    a2 = O.macro(p, f)[1][:, 0] @ np.sin(2 * math.pi * y / L)
    k = 2 * math.pi / L
    nu_meas = -math.log(a2 / a1) / (k * k * 300)
    assert abs(nu_meas / nu_expect - 1) < 3e-3


def test_threaded_build_gives_the_same_bits():
    """The OpenMP build of the oracle (nodes shared among threads) computes
    every node as the serial build does: same bits after 40 steps of a
    droplet, also with the test-only walls and a body force."""
    import lbm_inputs as I
    from oracle import analysis as An
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=-0.85, kappa=0.3)
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, 0.7 * Tc)
    rg, rl, _ = An.maxwell(p)
    rho0 = I.droplet_density(70, 46, 12, rl, rg)
    f1 = O.init_equilibrium(rho0)
    f4 = f1.copy()
    O.step(p, f1, 40)
    O.step(p, f4, 40, threads=4)
    assert np.array_equal(f1, f4)
    w = O.Params(G=0.0, walls_y=True, fext_x=1e-5, s=[1.0] * 9)
    g1 = O.init_equilibrium(np.ones((12, 9)))
    g4 = g1.copy()
    O.step(w, g1, 30)
    O.step(w, g4, 30, threads=3)
    assert np.array_equal(g1, g4)
