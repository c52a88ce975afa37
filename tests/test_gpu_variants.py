"""GPU-vs-oracle parity of the model variants: the Peng-Robinson law
(Eq. 29), the density-dependent shear viscosity of Section 4.2, Li et al.'s
third source entry (Eq. 26 note), and the BGK limit (all rates equal)."""
import warnings

import numpy as np
import pytest

import lbm_inputs as I
import oracle as O

warnings.filterwarnings("ignore", category=Warning, module="scipy")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_7228_gb300 as P
    P.lib()
    return P


def _run(P, prec, eos, op, rho0, steps, rho_ref, visc=None, sched=0, tile=0):
    ny, nx = rho0.shape
    lat = P.Lattice(nx, ny, prec)
    if sched or tile:
        lat.set_schedule(tile, sched)
    lat.set_params(eos, op.A, op.kappa, G=op.G, s=op.s, rho_ref=rho_ref, flags=P.LBM_FLAG_LI_EPS if op.li_eps else 0)
    if visc:
        lat.set_viscosity(*visc)
    lat.init_density(rho0)
    lat.step(steps)
    f = lat.read_populations()
    lat.close()
    return f


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _pr(P, kappa=0.3, s=(1.0,) * 9):
    from paper_1412_7228_gb300 import experiments as E
    eos = E.pr_eos()
    op = O.Params(eos=O.EOS_PR, a=eos.a, b=eos.b, R=eos.R, K=eos.K, T=eos.T, omega=eos.omega, Tc=eos.Tc, A=-0.3,
                  kappa=kappa, s=list(s))
    return eos, op


@pytest.mark.parametrize("prec,tol", [(2, 1e-12), (1, 2e-5)])
def test_peng_robinson_matches_oracle(P, prec, tol):
    eos, op = _pr(P)
    rho0 = I.droplet_density(80, 72, 18, 7.17, 0.0372, width=4.0)
    f = O.init_equilibrium(rho0)
    O.step(op, f, 60)
    assert _rel(_run(P, prec, eos, op, rho0, 60, 0.0372), f) <= tol


@pytest.mark.parametrize("prec,tol", [(2, 1e-12), (1, 2e-5)])
def test_density_dependent_viscosity_matches_oracle(P, prec, tol):
    eos, op = _pr(P, kappa=-1.0)
    op.var_visc, op.nu_g, op.nu_l, op.visc_rho_g, op.visc_rho_l = True, 0.2, 0.05, 0.0167, 7.17
    rho0 = I.ellipse_density(96, 96, 30, 27, 7.17, 0.0167, width=4.0)
    f = O.init_equilibrium(rho0)
    O.step(op, f, 60)
    assert _rel(_run(P, prec, eos, op, rho0, 60, 0.0167, visc=(0.2, 0.05, 0.0167, 7.17)), f) <= tol


@pytest.mark.parametrize("prec,tol", [(2, 1e-12), (1, 2e-5)])
def test_li_third_source_entry_matches_oracle(P, prec, tol):
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = 0.7 * Tc
    rg, rl, _ = P.lbm_eos_maxwell(eos)
    op = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=eos.T, A=-0.85, kappa=0.5, li_eps=True,
                  s=[1.0, 1.2, 1.3, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0])
    rho0 = I.droplet_density(70, 64, 14, rl, rg)
    f = O.init_equilibrium(rho0)
    O.step(op, f, 50)
    got = _run(P, prec, eos, op, rho0, 50, rg)
    assert _rel(got, f) <= tol
    op.li_eps = False
    g0 = O.init_equilibrium(rho0)
    O.step(op, g0, 50)
    assert _rel(g0, f) > 10 * tol            # the variant is not a no-op


def test_bgk_limit_equal_rates(P):
    """All rates equal to 1/tau: the MRT update is the BGK one; GPU and oracle
    agree, and the oracle's collision equals the textbook BGK-Guo formula."""
    omega = 1.0 / 0.8
    op = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.066, A=-0.85, kappa=0.0, s=[omega] * 9)
    rng = np.random.default_rng(1)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    t = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    for _ in range(5):
        f = t * 0.3 * rng.uniform(0.9, 1.1, 9)
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        rho = f.sum()
        ux = ((f * ex).sum() + Fx / 2) / rho
        uy = ((f * ey).sum() + Fy / 2) / rho
        eu = ex * ux + ey * uy
        feq = t * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy))
        Fb = t * (3 * ((ex - ux) * Fx + (ey - uy) * Fy) + 9 * eu * (ex * Fx + ey * Fy))
        bgk = f - omega * (f - feq) + (1 - omega / 2) * Fb
        np.testing.assert_allclose(O.collide_node(op, f, Fx, Fy), bgk, rtol=0, atol=1e-15)
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.066)
    rho0 = I.droplet_density(48, 48, 10, 0.36, 0.0095)
    f = O.init_equilibrium(rho0)
    O.step(op, f, 40)
    assert _rel(_run(P, P.LBM_FP64, eos, op, rho0, 40, 0.0095), f) <= 1e-12


@pytest.mark.parametrize("prec", [2, 1])
def test_every_variant_gives_the_same_bits_in_every_schedule(P, prec):
    """The variants take the general path or other pressure laws in the
    fused kernels: the Peng-Robinson and van der Waals laws, the
    density-dependent viscosity, Li's source entry and G = 0.  One step per
    launch, the multi-step schedule and the cluster schedule, on tile shapes
    that do not divide the lattice, give the same bits for each."""
    from paper_1412_7228_gb300 import experiments as E
    eos_pr, op_pr = _pr(P)
    vdw = E.vdw_eos(0.9, 0.3)
    op_vdw = O.Params(eos=O.EOS_VDW, a=vdw.a, b=vdw.b, R=1.0, K=0.3, T=vdw.T, A=-0.5, kappa=0.5, s=[1.0] * 9)
    eos_v, op_v = _pr(P, kappa=-1.0)
    cs = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.066)
    op_li = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.066, A=-0.85, kappa=0.5, li_eps=True)
    op_g0 = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.066, A=-0.85, kappa=0.5, G=0.0)
    cases = [
        (eos_pr, op_pr, I.droplet_density(150, 70, 18, 7.17, 0.0372, width=4.0), 0.0372, None),
        (vdw, op_vdw, I.slab_density(150, 70, 5.8, 1.47, width=4.0), 1.47, None),
        (eos_v, op_v, I.ellipse_density(150, 70, 30, 20, 7.17, 0.0167, width=4.0), 0.0167, (0.2, 0.05, 0.0167, 7.17)),
        (cs, op_li, I.droplet_density(150, 70, 14, 0.36, 0.0095), 0.0095, None),
        (cs, op_g0, 0.3 + 0.01 * I.droplet_density(150, 70, 14, 1.0, 0.0), 0.3, None),
    ]
    for eos, op, rho0, rho_ref, visc in cases:
        base = _run(P, prec, eos, op, rho0, 23, rho_ref, visc)
        assert np.all(np.isfinite(base))
        assert np.array_equal(_run(P, prec, eos, op, rho0, 23, rho_ref, visc, sched=3), base), (op.eos, visc)
        # another tile shape in the multi-step schedule
        other = [k for k, c in enumerate(P.lbm_tile_configs(prec)) if c[3] == 1][-1]
        assert np.array_equal(_run(P, prec, eos, op, rho0, 23, rho_ref, visc, sched=3, tile=other), base), \
            (op.eos, visc, other)
        # the cluster schedule, on a 64 x 60 window around the lattice's centre
        # (the drop or ellipse whole inside, gas or liquid at its edges)
        w = np.ascontiguousarray(rho0[5:65, 43:107])
        ref = _run(P, prec, eos, op, w, 23, rho_ref, visc)
        assert np.array_equal(_run(P, prec, eos, op, w, 23, rho_ref, visc, sched=4), ref), (op.eos, visc, 4)
