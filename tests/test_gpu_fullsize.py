"""Parity at the benchmark's full size (4096x4096 spinodal), in the launch
configuration bench.py times (its default tiles, one tile per CTA, CUDA
graphs), on sampled outputs the oracle can compute one by one.

A node's state after n steps depends only on the initial field within 2n
nodes (the pull reaches one node, psi one more), so the oracle runs on a
window of the initial field around each sample and its interior (2n nodes
from the window's edge) is exact.  The window is extended by its mirror
images into a 2W x 2W periodic domain, so that its edges meet continuous
data: a liquid/gas jump across a seam would be stepped by the oracle like a
real interface and could leave the psi domain there.  Windows sit on the domain's
corners and edges (periodic wrap through the ghost cells), on tile seams and
at seeded random places.  Mass is checked as a property at full size."""
import warnings

import numpy as np
import pytest

import bench
import lbm_inputs as I
import oracle as O

warnings.filterwarnings("ignore", category=Warning, module="scipy")

pytestmark = pytest.mark.gpu

N = 4096
STEPS = 3
W = 24                      # oracle window edge
M = 2 * STEPS               # invalid margin inside a window
S_CFG = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_7228_gb300 as P
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = 0.7 * Tc
    op = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=eos.T, A=-0.85, kappa=0.3, s=list(S_CFG))
    rho0 = I.spinodal_density(N, N, 0.25, 0.01, 14127228)
    return P, eos, op, rho0


def _windows():
    rng = np.random.default_rng(4096)
    c = [(0, 0), (N - 1, N - 1), (0, N // 2), (N // 2, 0), (N - 1, 7), (127, 15), (128, 16), (255, 2047),
         (2048, 1023)]
    c += [tuple(int(v) for v in rng.integers(0, N, 2)) for _ in range(7)]
    return c


def _window(rho0, n, cx, cy):
    idx_x = (np.arange(W) + cx - W // 2) % n
    idx_y = (np.arange(W) + cy - W // 2) % n
    return idx_x, idx_y


def _oracle_on_window(op, rho0, idx_x, idx_y):
    """Density after STEPS oracle steps on the window, mirrored to 2W x 2W."""
    w = rho0[np.ix_(idx_y, idx_x)]
    top = np.concatenate([w, w[:, ::-1]], axis=1)
    dom = np.ascontiguousarray(np.concatenate([top, top[::-1, :]], axis=0))
    f = O.init_equilibrium(dom)
    O.step(op, f, STEPS)
    return O.macro(op, f)[0][:W, :W]


def _oracle_window(op, rho0, cx, cy):
    idx_x, idx_y = _window(rho0, N, cx, cy)
    return _oracle_on_window(op, rho0, idx_x, idx_y), idx_x, idx_y


@pytest.mark.parametrize("prec,cfg,tol", [(1, bench.TILE_FP32, 1e-6), (2, bench.TILE_FP64, 1e-13)])
def test_bench_configuration_matches_oracle_on_sampled_windows(setup, prec, cfg, tol):
    P, eos, op, rho0 = setup
    lat = P.Lattice(N, N, prec)
    lat.set_schedule(cfg, 0)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=0.25)
    lat.init_density(rho0)
    lat.use_graphs(True)
    lat.step(STEPS)
    rho = lat.read_fields(which=("rho",))["rho"]
    lat.close()
    worst = 0.0
    for cx, cy in _windows():
        ref, ix, iy = _oracle_window(op, rho0, cx, cy)
        got = rho[np.ix_(iy, ix)]
        inner = (slice(M, W - M), slice(M, W - M))
        worst = max(worst, float(np.abs(got[inner] / ref[inner] - 1).max()))
    assert worst <= tol, worst


def test_bench_configuration_conserves_mass(setup):
    P, eos, op, rho0 = setup
    lat = P.Lattice(N, N, P.LBM_FP32)
    lat.set_schedule(bench.TILE_FP32, 0)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=0.25)
    lat.init_density(rho0)
    lat.use_graphs(True)
    m0 = lat.stats()["mass"]
    lat.step(256)
    st = lat.stats()
    lat.close()
    assert abs(st["mass"] / m0 - 1) < 1e-7
    assert abs(st["mom_x"]) < 1e-6 * m0 and abs(st["mom_y"]) < 1e-6 * m0


@pytest.mark.parametrize("prec,tol,sched", [(1, 2e-6, None), (2, 1e-14, None), (1, 2e-6, 3)])
def test_batched_sweep_configuration_matches_oracle_on_sampled_windows(setup, prec, tol, sched):
    """The 64 uneven droplets of the batched sweep (L in {128, ..., 1024},
    seed 7228) in one batched launch, tile shape autotuned and graphs on
    as the sweep runs them (or in the multi-step schedule: one launch per
    chunk of at most 32 instances and 64 MiB of populations): 3 steps, then three oracle
    windows per instance (on the interface, across the wrapped corner, at a
    seeded place).
    Error: max |rho - rho_oracle| over a window / max rho_oracle there.  A
    gas node next to the interface receives populations of liquid size, so
    its error scales with the liquid density, not its own: in FP32 (unit
    roundoff 6e-8, about 30 roundings per population and step) 3 steps stay
    below 2e-6 of the window's largest density."""
    P = setup[0]
    from paper_1412_7228_gb300 import sweep
    drops = sweep.sweep_droplets()
    b = P.Batch([d.L for d in drops], [d.L for d in drops], prec)
    cases = []
    for i, d in enumerate(drops):
        eos, rg, rl = sweep.cs_eos(d.t_over_tc)
        rho0 = I.droplet_density(d.L, d.L, d.radius, rl, rg)
        b.set_params(i, eos, d.A, d.kappa, G=-1.0, s=S_CFG, rho_ref=rg)
        b.init_density(i, rho0)
        op = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=eos.T, A=d.A, kappa=d.kappa, s=list(S_CFG))
        cases.append((d, op, rho0))
    if sched is None:
        b.autotune(3)
    else:
        b.set_schedule(0, sched)
    b.use_graphs(True)
    b.step(STEPS)
    rng = np.random.default_rng(7228)
    worst = 0.0
    for i, (d, op, rho0) in enumerate(cases):
        assert b.status(i) == 0
        rho = b.read_fields(i, which=("rho",))["rho"]
        n = d.L
        for cx, cy in ((int(n / 2 + d.radius), n // 2), (0, 0), tuple(int(v) for v in rng.integers(0, n, 2))):
            ix, iy = _window(rho0, n, cx, cy)
            ref = _oracle_on_window(op, rho0, ix, iy)[M:W - M, M:W - M]
            got = rho[np.ix_(iy, ix)][M:W - M, M:W - M]
            worst = max(worst, float(np.abs(got - ref).max() / ref.max()))
    b.close()
    assert worst <= tol, worst
