"""GPU-vs-oracle parity of the fused sm_103a step, through the C ABI.

Tolerances, from the arithmetic of the two paths:
  FP64: the kernel evaluates the same formulas in a different order (unrolled
        moments, fused multiply-adds); after n steps of a dissipative update
        the populations agree to ~1e-15 n relative -> 1e-12 for n <= 100.
  FP32: populations are stored as deviations from t_a rho_ref and updated in
        FP32 (unit roundoff 6e-8); about 30 roundings feed each population per
        step and errors of a stable step do not grow, so 50 steps stay within
        2e-5 of the largest population; density fields within 1e-4 relative.
"""
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
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_7228_gb300 as P
    P.lib()
    return P


def cs_case(P, tr=0.7, A=-0.85, kappa=0.3):
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = tr * Tc
    rg, rl, _ = P.lbm_eos_maxwell(eos)
    op = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=eos.T, A=A, kappa=kappa, G=-1.0, s=list(S_CFG))
    return eos, op, rg, rl


def oracle_run(op, rho0, steps):
    f = O.init_equilibrium(rho0)
    O.step(op, f, steps)
    return f


def gpu_run(P, prec, eos, op, rho0, steps, rho_ref, cfg=None, sched=0, graphs=False):
    ny, nx = rho0.shape
    lat = P.Lattice(nx, ny, prec)
    if cfg is not None:
        lat.set_schedule(cfg, sched)
    lat.set_params(eos, op.A, op.kappa, G=op.G, s=op.s, rho_ref=rho_ref)
    lat.init_density(rho0)
    if graphs:
        lat.use_graphs(True)
    lat.step(steps)
    lat.sync()
    f = lat.read_populations()
    lat.close()
    return f


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec,tol", [(2, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("shape", [(100, 70), (64, 64), (130, 36)])
def test_droplet_populations_match_oracle(P, prec, tol, shape):
    """Several tiles and ragged tails in x and y, 50 steps."""
    nx, ny = shape
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(nx, ny, min(nx, ny) / 4, rl, rg)
    ref = oracle_run(op, rho0, 50)
    got = gpu_run(P, prec, eos, op, rho0, 50, rho_ref=rg)
    assert rel(got, ref) <= tol


@pytest.mark.parametrize("shape", [(4, 4), (6, 6), (8, 5), (2, 2), (3, 7), (33, 17)])
def test_tiny_and_odd_domains(P, shape):
    nx, ny = shape
    eos, op, rg, rl = cs_case(P, kappa=0.5)
    rho0 = I.spinodal_density(nx, ny, rho0=0.25, amp=0.05, seed=nx * 131 + ny)
    ref = oracle_run(op, rho0, 10)
    assert rel(gpu_run(P, P.LBM_FP64, eos, op, rho0, 10, rho_ref=0.25), ref) <= 1e-12
    assert rel(gpu_run(P, P.LBM_FP32, eos, op, rho0, 10, rho_ref=0.25), ref) <= 2e-5


def test_every_tile_config_and_graphs_are_bit_identical(P):
    """The per-node arithmetic does not depend on the tiling: every tile
    configuration, CTA schedule and the CUDA-graph path give the same bits."""
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(90, 75, 20, rl, rg)
    for prec in (P.LBM_FP64, P.LBM_FP32):
        base = gpu_run(P, prec, eos, op, rho0, 70, rho_ref=rg, cfg=0)
        for k, c in enumerate(P.lbm_tile_configs(prec)):
            assert np.array_equal(gpu_run(P, prec, eos, op, rho0, 70, rho_ref=rg, cfg=k), base), (prec, k)
            if c[3] == 1:   # the multi-step persistent launch of the same tiles
                assert np.array_equal(gpu_run(P, prec, eos, op, rho0, 70, rho_ref=rg, cfg=k, sched=3), base), \
                    (prec, k, 3)
        assert np.array_equal(gpu_run(P, prec, eos, op, rho0, 70, rho_ref=rg, graphs=True), base)


def test_graph_replays_of_every_length_give_the_one_step_bits(P):
    """With graphs on, lbm_step(n) replays graphs of 32, 16, 8, 4 and 2 steps
    (the binary digits of n below 32) and launches an odd last step plainly:
    every split of the steps into calls, with the graphs captured ahead
    (capture_graphs) or on first use, gives the bits of plain launches and
    counts one kernel launch per step."""
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(90, 75, 20, rl, rg)
    counts = (1, 2, 3, 5, 20, 37, 64, 6)
    base = gpu_run(P, P.LBM_FP32, eos, op, rho0, sum(counts), rho_ref=rg)
    for ahead in (False, True):
        lat = P.Lattice(90, 75, P.LBM_FP32)
        lat.set_params(eos, op.A, op.kappa, G=op.G, s=op.s, rho_ref=rg)
        lat.init_density(rho0)
        lat.use_graphs(True)
        if ahead:
            lat.capture_graphs()
        n0 = lat.kernel_launches
        for n in counts:
            lat.step(n)
        assert lat.kernel_launches - n0 == sum(counts) and lat.steps_done == sum(counts)
        lat.sync()
        assert np.array_equal(lat.read_populations(), base), ahead
        lat.close()
    lat = P.Lattice(90, 75, P.LBM_FP32)   # graphs off or the multi-step schedule: nothing to capture
    lat.set_params(eos, op.A, op.kappa, G=op.G, s=op.s, rho_ref=rg)
    lat.init_density(rho0)
    lat.capture_graphs()
    lat.use_graphs(True)
    lat.set_schedule(0, 3)
    lat.capture_graphs()
    lat.close()


def test_cluster_schedule_gives_the_one_step_bits(P):
    """Schedule 4 holds a single lattice in the shared memory of one
    thread-block cluster (strips of rows per CTA, edge rows exchanged through
    distributed shared memory, one cluster barrier per step): the one-step
    bits for lattices of one CTA up to sixteen, ragged last strips, the fast
    and the general path, however the steps are split into calls; refused
    for a batch and for lattices it cannot hold."""
    eos, op, rg, rl = cs_case(P)
    shapes = {P.LBM_FP32: [(64, 64), (100, 100), (128, 128), (90, 75), (33, 18), (8, 5), (50, 2)],
              P.LBM_FP64: [(64, 64), (40, 30), (8, 5), (50, 100)]}
    for prec, cases in shapes.items():
        for nx, ny in cases:
            rho0 = I.droplet_density(nx, ny, min(nx, ny) / 4, rl, rg)
            base = gpu_run(P, prec, eos, op, rho0, 37, rho_ref=rg)
            lat = P.Lattice(nx, ny, prec)
            lat.set_schedule(0, 4)
            lat.set_params(eos, op.A, op.kappa, G=op.G, s=op.s, rho_ref=rg)
            lat.init_density(rho0)
            lat.use_graphs(True)
            n0 = lat.kernel_launches
            for n in (1, 0, 7, 29):
                lat.step(n)
            assert lat.kernel_launches - n0 == 3 and lat.steps_done == 37
            lat.sync()
            assert np.array_equal(lat.read_populations(), base), (prec, nx, ny)
            assert np.array_equal(lat.read_fields(which=("rho",))["rho"],
                                  gpu_fields(P, prec, eos, op, rho0, 37, rg)), (prec, nx, ny)
            lat.close()
    for prec, (nx, ny) in ((P.LBM_FP32, (200, 50)), (P.LBM_FP32, (64, 17)), (P.LBM_FP64, (100, 40))):
        lat = P.Lattice(nx, ny, prec)
        with pytest.raises(P.LbmError) as ei:
            lat.set_schedule(0, 4)
        assert ei.value.code == -1
        lat.close()
    b = P.Batch([32, 32], [32, 32], P.LBM_FP32)
    with pytest.raises(P.LbmError):
        b.set_schedule(0, 4)
    b.close()


def gpu_fields(P, prec, eos, op, rho0, steps, rho_ref):
    ny, nx = rho0.shape
    lat = P.Lattice(nx, ny, prec)
    lat.set_params(eos, op.A, op.kappa, G=op.G, s=op.s, rho_ref=rho_ref)
    lat.init_density(rho0)
    lat.step(steps)
    rho = lat.read_fields(which=("rho",))["rho"]
    lat.close()
    return rho


def test_multi_step_launch_in_pieces_and_tiny_lattices(P):
    """The multi-step schedule gives the one-step bits however the steps are
    split into calls (odd counts flip the time level inside a launch), on a
    lattice of a single tile (the tile is its own periodic neighbourhood) and
    on ones whose tiles do not divide them, and on one whose last tile column
    and row are one node wide (the tiles on either side of them depend on each
    other), with graphs requested (not used); in two tile shapes."""
    eos, op, rg, rl = cs_case(P)
    for nx, ny in ((64, 16), (90, 75), (200, 37), (257, 49), (20, 49)):
        rho0 = I.droplet_density(nx, ny, min(nx, ny) / 4, rl, rg)
        for prec, tile in [(p, k) for p in (P.LBM_FP64, P.LBM_FP32)
                           for k in [0] + [k for k, c in enumerate(P.lbm_tile_configs(p)) if c[3] == 1][-1:]]:
            base = gpu_run(P, prec, eos, op, rho0, 37, rho_ref=rg)
            lat = P.Lattice(nx, ny, prec)
            lat.set_schedule(tile, 3)
            lat.set_params(eos, op.A, op.kappa, G=op.G, s=op.s, rho_ref=rg)
            lat.init_density(rho0)
            lat.use_graphs(True)
            n0 = lat.kernel_launches
            for n in (1, 0, 7, 29):
                lat.step(n)
            assert lat.kernel_launches - n0 == 3 and lat.steps_done == 37
            lat.sync()
            assert np.array_equal(lat.read_populations(), base), (nx, ny, prec, tile)
            lat.close()


def test_vdw_flat_interface_matches_oracle_and_table1(P, golden):
    """The paper's flat-interface case (Table 1) on the GPU in FP64: same
    populations as the oracle after 2000 steps, and after 15000 steps the
    printed densities to all digits (s = 1, reading R14)."""
    eos = P.Eos(kind=P.LBM_EOS_VDW, a=9 / 49, b=2 / 21, R=1.0, K=0.3)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = 0.9 * Tc
    op = O.Params(eos=O.EOS_VDW, a=9 / 49, b=2 / 21, R=1.0, K=0.3, T=eos.T, A=-0.5, kappa=0.5, s=[1.0] * 9)
    rho0 = I.slab_density(128, 4, 5.8, 1.47, width=4.0)
    ref = oracle_run(op, rho0, 2000)
    assert rel(gpu_run(P, P.LBM_FP64, eos, op, rho0, 2000, rho_ref=1.47), ref) <= 1e-11
    lat = P.Lattice(128, 4, P.LBM_FP64)
    lat.set_params(eos, -0.5, 0.5, G=-1.0, s=[1.0] * 9, rho_ref=1.47)
    lat.init_density(rho0)
    lat.step(15000)
    rho = lat.read_fields(which=("rho",))["rho"]
    rl, rg = An.slab_densities(rho)
    t1 = golden["table1_flat_interface"]
    assert round(rl, 5) == t1["rho_l"] and round(rg, 5) == t1["rho_g"]


def test_static_droplet_64_after_10000_steps(P):
    """64x64 Carnahan-Starling droplet, R = 15, T = 0.7 Tc, kappa = 0,
    10^4 steps: density max relative error <= 1e-10 (FP64), <= 1e-4 (FP32)."""
    eos, op, rg, rl = cs_case(P, kappa=0.0)
    rho0 = I.droplet_density(64, 64, 15, rl, rg)
    f_ref = oracle_run(op, rho0, 10000)
    rho_ref_field = O.macro(op, f_ref)[0]
    for prec, tol in ((P.LBM_FP64, 1e-10), (P.LBM_FP32, 1e-4)):
        lat = P.Lattice(64, 64, prec)
        lat.set_params(eos, op.A, 0.0, s=S_CFG, rho_ref=rg)
        lat.init_density(rho0)
        lat.step(10000)
        rho = lat.read_fields(which=("rho",))["rho"]
        lat.close()
        err = float(np.abs(rho / rho_ref_field - 1).max())
        assert err <= tol, (prec, err)


@pytest.mark.parametrize("prec,tol", [(2, 1e-10), (1, 1e-4)])
def test_fields_measure_and_stats_match_oracle(P, prec, tol):
    eos, op, rg, rl = cs_case(P)
    nx, ny = 80, 64
    rho0 = I.droplet_density(nx, ny, 16, rl, rg)
    f_ref = oracle_run(op, rho0, 300)
    r, ux, uy, psi, Fx, Fy = O.macro(op, f_ref)
    lat = P.Lattice(nx, ny, prec)
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    lat.step(300)
    fl = lat.read_fields()
    assert rel(fl["rho"], r) <= tol and rel(fl["psi"], psi) <= tol
    umax = np.hypot(ux, uy).max()
    assert np.abs(fl["ux"] - ux).max() <= 100 * tol * umax + 1e-12
    m = lat.measure_pressure_jump(nx / 2, ny / 2, 8, 24)
    d = An.pressure_jump(op, r, nx / 2, ny / 2, 8, 24)
    for k in ("p_in", "p_out", "rho_in", "rho_out", "R_eq"):
        assert abs(m[k] / d[k] - 1) <= tol, k
    st = lat.stats()
    assert abs(st["mass"] / r.sum() - 1) <= tol
    assert abs(st["umax"] / umax - 1) <= 100 * tol
    assert abs(st["ke"] / (0.5 * r * (ux * ux + uy * uy)).sum() - 1) <= 100 * tol
    lat.close()


def test_g_zero_shear_wave_matches_oracle(P):
    """G = 0: no psi, F = Q = 0 (reading R11)."""
    L = 64
    y = np.arange(L)
    ux = np.broadcast_to((1e-3 * np.sin(2 * np.pi * y / L))[:, None], (L, 32)).copy()
    op = O.Params(G=0.0, s=[1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1.3, 1.3], eos=O.EOS_CS, a=1, b=4, R=1, K=1, T=0.07)
    f = O.init_equilibrium(np.ones((L, 32)), ux, np.zeros_like(ux))
    O.step(op, f, 200)
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1, b=4, R=1, K=1, T=0.07)
    lat = P.Lattice(32, L, P.LBM_FP64)
    lat.set_params(eos, op.A, 0.0, G=0.0, s=op.s, rho_ref=1.0)
    lat.init_density(np.ones((L, 32)), ux, np.zeros_like(ux))
    lat.step(200)
    assert rel(lat.read_populations(), f) <= 1e-12
    lat.close()


def test_batch_equals_separate_runs(P):
    """Uneven instances stepped together in one launch per step give the
    same bits as each instance alone, for every CTA schedule."""
    eos, op, rg, rl = cs_case(P)
    shapes = [(96, 96), (40, 72), (130, 50)]
    rhos = [I.droplet_density(nx, ny, min(nx, ny) / 4, rl, rg) for nx, ny in shapes]
    for prec in (P.LBM_FP64, P.LBM_FP32):
        solo = [gpu_run(P, prec, eos, op, r, 40, rho_ref=rg) for r in rhos]
        for sched in (0, 1, 2, 3):
            b = P.Batch([s[0] for s in shapes], [s[1] for s in shapes], prec)
            b.set_schedule(0, sched)
            for i, r in enumerate(rhos):
                b.set_params(i, eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
                b.init_density(i, r)
            b.step(40)
            outs = [b.read_populations(i) for i in range(len(shapes))]
            b.close()
            for i in range(len(shapes)):
                assert np.array_equal(outs[i], solo[i]), (prec, sched, i)


def test_batch_of_more_than_64_instances(P):
    """A batch beyond one launch's 64 instances (70 uneven lattices: two
    launches per step) gives every instance the bits it gets alone, for each
    CTA schedule, in the one-tile-per-CTA and the persistent tile shapes, with
    CUDA graphs, and counts two kernel launches per step (the multi-step
    schedule: one launch per 32 instances for all the steps)."""
    eos, op, rg, rl = cs_case(P)
    rng = np.random.default_rng(70)
    shapes = [(int(rng.integers(16, 48)), int(rng.integers(24, 56))) for _ in range(70)]
    rhos = [I.droplet_density(nx, ny, min(nx, ny) / 4, rl, rg) for nx, ny in shapes]
    steps = 40
    solo = [gpu_run(P, P.LBM_FP32, eos, op, r, steps, rho_ref=rg) for r in rhos]
    persistent = [k for k, c in enumerate(P.lbm_tile_configs(P.LBM_FP32)) if c[3] == 2]
    runs = [(c, s) for c in (0, persistent[0]) for s in (0, 1, 2)]
    runs += [(k, 3) for k, c in enumerate(P.lbm_tile_configs(P.LBM_FP32)) if c[3] == 1]
    for cfg, sched in runs:
        b = P.Batch([s[0] for s in shapes], [s[1] for s in shapes], P.LBM_FP32)
        b.set_schedule(cfg, sched)
        for i, r in enumerate(rhos):
            b.set_params(i, eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
            b.init_density(i, r)
        b.use_graphs(True)
        n0 = b.kernel_launches
        b.step(steps)
        # one launch per step and 64 instances; the multi-step schedule one launch per 32
        assert b.kernel_launches - n0 == (3 if sched == 3 else 2 * steps)
        outs = [b.read_populations(i) for i in range(len(shapes))]
        b.close()
        for i in range(len(shapes)):
            assert np.array_equal(outs[i], solo[i]), (cfg, sched, i)


def test_multi_step_chunks_of_mixed_sizes_give_the_solo_bits(P):
    """The multi-step schedule's chunking on a batch of mixed sizes: a lattice
    whose populations exceed a chunk's budget (a chunk of its own), lattices
    sorted largest first and spread over even chunks, and thin ones (one
    tile column; a last tile row one node high): every instance gets the
    bits it gets alone."""
    eos, op, rg, rl = cs_case(P)
    shapes = [(64, 64), (2100, 2100), (300, 20), (17, 1000), (64, 64), (900, 700), (1000, 17), (64, 64)]
    rhos = [I.spinodal_density(nx, ny, rho0=0.25, amp=0.01, seed=nx * 7 + ny) for nx, ny in shapes]
    steps = 12
    solo = [gpu_run(P, P.LBM_FP32, eos, op, r, steps, rho_ref=0.25) for r in rhos]
    b = P.Batch([s_[0] for s_ in shapes], [s_[1] for s_ in shapes], P.LBM_FP32)
    b.set_schedule(0, 3)
    for i, r in enumerate(rhos):
        b.set_params(i, eos, op.A, op.kappa, s=S_CFG, rho_ref=0.25)
        b.init_density(i, r)
    n0 = b.kernel_launches
    b.step(5)
    b.step(7)
    launches = b.kernel_launches - n0
    outs = [b.read_populations(i) for i in range(len(shapes))]
    b.close()
    # one launch per chunk of the host plan, the same chunks for both calls
    plan = P.lbm_run_chunk_plan([s_[0] for s_ in shapes], [s_[1] for s_ in shapes], P.LBM_FP32)
    assert launches == 2 * (max(plan) + 1) and max(plan) + 1 >= 2
    for i in range(len(shapes)):
        assert np.array_equal(outs[i], solo[i]), (i, shapes[i])


def test_checkpoint_resume_is_bit_identical(P, tmp_path):
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(70, 50, 12, rl, rg)
    path = str(tmp_path / "ck.bin")
    lat = P.Lattice(70, 50, P.LBM_FP32)
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    lat.step(25)
    lat.save(path)
    lat.step(25)
    straight = lat.read_populations()
    lat.close()
    lat2 = P.Lattice(70, 50, P.LBM_FP32)
    lat2.load(path)
    assert lat2.steps_done == 25
    lat2.step(25)
    assert np.array_equal(lat2.read_populations(), straight)
    lat2.close()


@pytest.mark.parametrize("graphs", [False, True])
def test_autotune_keeps_the_state(P, graphs):
    """Timing every tile and schedule (with graphs: over captured graph
    replays) leaves the state, step count and results untouched."""
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(128, 96, 20, rl, rg)
    ref = gpu_run(P, P.LBM_FP32, eos, op, rho0, 30, rho_ref=rg)
    lat = P.Lattice(128, 96, P.LBM_FP32)
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    lat.use_graphs(graphs)
    k, s, ms = lat.autotune(5)
    assert 0 <= k < len(P.lbm_tile_configs(P.LBM_FP32)) and s in (0, 3, 4) and ms > 0
    assert lat.steps_done == 0
    lat.step(30)
    assert np.array_equal(lat.read_populations(), ref)
    lat.close()


def test_density_outside_psi_domain_reports_unstable(P):
    """R18: a density beyond the EOS's psi domain is reported, not clamped."""
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(32, 32, 6, rl, rg)
    rho0[16, 16] = 0.7            # rho/3 - p_EOS < 0 for the CS law here
    lat = P.Lattice(32, 32, P.LBM_FP32)
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    lat.step(1)
    with pytest.raises(P.LbmError) as ei:
        lat.sync()
    assert ei.value.code == -4
    lat.close()


def test_nan_initial_field_is_rejected(P):
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(16, 16, 4, rl, rg)
    rho0[3, 3] = np.nan
    lat = P.Lattice(16, 16, P.LBM_FP32)
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
    with pytest.raises(P.LbmError) as ei:
        lat.init_density(rho0)
    assert ei.value.code == -1
    lat.close()


@pytest.mark.parametrize("sched,other", [(0, False), (3, False), (3, True)])
def test_bounded_wait_reports_timeout_and_context_survives(P, sched, other):
    """A barrier phase nothing completes: every CTA gives up after its
    limit, the status reads ETIMEOUT, and the context keeps working (in the
    multi-step launch the CTA that gives up raises the launch's abort flag
    and the other CTAs stop at their next work item)."""
    eos, op, rg, rl = cs_case(P)
    rho0 = I.droplet_density(64, 32, 8, rl, rg)
    lat = P.Lattice(64, 32, P.LBM_FP32)
    tile = [k for k, c in enumerate(P.lbm_tile_configs(P.LBM_FP32)) if c[3] == 1][-1] if other else 0
    lat.set_schedule(tile, sched)
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg, flags=P.LBM_FLAG_TEST_FORCE_TIMEOUT)
    lat.init_density(rho0)
    lat.step(1 if sched == 0 else 5)
    with pytest.raises(P.LbmError) as ei:
        lat.sync()
    assert ei.value.code == -5
    lat.clear_status()
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg, flags=0)
    lat.init_density(rho0)
    lat.step(10)
    lat.sync()
    ref = oracle_run(op, rho0, 10)
    assert rel(lat.read_populations(), ref) <= 2e-5
    lat.close()


def test_autotune_passes_over_pairs_whose_waits_gave_up(P):
    """Every bounded wait forced to give up: no (tile, schedule) pair of a
    batch is left, so the autotuner reports ETIMEOUT and puts back the
    populations, the step count and the schedule it found (here the
    multi-step one: one launch per call); stepping afterwards gives the bits
    of a batch that was never tuned."""
    eos, op, rg, rl = cs_case(P)
    shapes = [(64, 32), (48, 40)]
    rho = [I.droplet_density(nx, ny, 8, rl, rg) for nx, ny in shapes]

    def make(flags):
        b = P.Batch([s[0] for s in shapes], [s[1] for s in shapes], P.LBM_FP32)
        b.set_schedule(0, 3)
        for i, r in enumerate(rho):
            b.set_params(i, eos, op.A, op.kappa, s=S_CFG, rho_ref=rg, flags=flags)
            b.init_density(i, r)
        return b

    b = make(P.LBM_FLAG_TEST_FORCE_TIMEOUT)
    before = [b.read_populations(i) for i in range(len(shapes))]
    with pytest.raises(P.LbmError) as ei:
        b.autotune(2)
    assert ei.value.code == -5
    assert b.steps_done == 0
    for i in range(len(shapes)):
        assert np.array_equal(b.read_populations(i), before[i])
        b.set_params(i, eos, op.A, op.kappa, s=S_CFG, rho_ref=rg, flags=0)
    n0 = b.kernel_launches
    b.step(7)
    b.sync()
    assert b.kernel_launches - n0 == 1 and b.steps_done == 7
    ref = make(0)
    ref.step(7)
    ref.sync()
    for i in range(len(shapes)):
        assert np.array_equal(b.read_populations(i), ref.read_populations(i))
    b.close()
    ref.close()


def test_symmetric_droplet_stays_bitwise_mirror_symmetric(P):
    """Rounding of the FP32 path respects the lattice mirrors: a centred drop
    stays symmetric to the last bit, so it cannot drift off its centre."""
    eos, op, rg, rl = cs_case(P, kappa=0.3)
    n = 64
    rho0 = I.droplet_density(n, n, 15, rl, rg)
    lat = P.Lattice(n, n, P.LBM_FP32)
    lat.set_params(eos, op.A, op.kappa, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    lat.step(2000)
    f = lat.read_populations()
    lat.close()
    mx = [0, 3, 2, 1, 4, 6, 5, 8, 7]          # x -> -x
    my = [0, 1, 4, 3, 2, 8, 7, 6, 5]          # y -> -y
    xs = (-np.arange(n)) % n
    for a in range(9):
        assert np.array_equal(f[a], f[mx[a]][:, xs]), a
        assert np.array_equal(f[a], f[my[a]][xs, :]), a
