"""Argument checks, allocation failure and a lattice whose population arrays
exceed 2^31 elements, on the GPU.  Every rejected call returns its error code,
creates nothing, and leaves an existing context usable."""
import ctypes
import warnings

import numpy as np
import pytest

import lbm_inputs as I
import oracle as O

warnings.filterwarnings("ignore", category=Warning, module="scipy")

pytestmark = pytest.mark.gpu
S_CFG = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_7228_gb300 as P
    return P


def _cs(P):
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = 0.7 * Tc
    op = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=eos.T, A=-0.85, kappa=0.3, s=list(S_CFG))
    rg, rl, _ = P.lbm_eos_maxwell(eos)
    return eos, op, rg, rl


def _create(P, nx, ny, prec, buf=None, nbytes=0):
    ctx = ctypes.c_void_p()
    rc = P.lbm.lib().lbm_create(ctypes.byref(ctx), nx, ny, prec, buf, nbytes, None)
    return rc, ctx


def test_shapes_and_precisions_are_checked(P):
    for nx, ny, prec in ((1, 8, 1), (8, 1, 1), (0, 0, 1), (-4, 8, 1), ((1 << 20) + 1, 8, 1), (8, 8, 3), (8, 8, 0)):
        rc, ctx = _create(P, nx, ny, prec)
        assert rc == P.lbm.LBM_EINVAL and not ctx.value, (nx, ny, prec)


def test_allocation_failure_is_an_error_code(P):
    """2^20 x 2^20 nodes need about 80 TB: the allocation fails cleanly."""
    rc, ctx = _create(P, 1 << 20, 1 << 20, P.LBM_FP32)
    assert rc == P.lbm.LBM_ENOMEM and not ctx.value


def test_caller_buffer_is_checked(P):
    import torch
    need = P.lbm_required_bytes(64, 64, P.LBM_FP32)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    rc, ctx = _create(P, 64, 64, P.LBM_FP32, ctypes.c_void_p(base), need - 256)
    assert rc == P.lbm.LBM_ENOMEM and not ctx.value
    rc, ctx = _create(P, 64, 64, P.LBM_FP32, ctypes.c_void_p(base + 16), need)
    assert rc == P.lbm.LBM_EINVAL and not ctx.value
    rc, ctx = _create(P, 64, 64, P.LBM_FP32, ctypes.c_void_p(base), need)
    assert rc == P.lbm.LBM_OK and ctx.value
    P.lbm.lib().lbm_destroy(ctx)


def test_rejected_calls_leave_the_context_usable(P):
    eos, op, rg, rl = _cs(P)
    lat = P.Lattice(40, 36, P.LBM_FP32)
    with pytest.raises(P.LbmError) as ei:
        lat.step(1)                                   # parameters never set
    assert ei.value.code == P.lbm.LBM_EINVAL
    bad = [dict(s=[1.0] * 8 + [2.0]), dict(s=[0.0] + [1.0] * 8), dict(s=[1.0] * 8 + [float("nan")])]
    for kw in bad:
        with pytest.raises(P.LbmError) as ei:
            lat.set_params(eos, -0.85, 0.3, rho_ref=rg, **kw)
        assert ei.value.code == P.lbm.LBM_EINVAL
    cold = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.0)
    with pytest.raises(P.LbmError):
        lat.set_params(cold, -0.85, 0.3, rho_ref=rg)
    with pytest.raises(P.LbmError):
        lat.set_params(eos, float("inf"), 0.3, rho_ref=rg)
    rc = P.lbm.lib().lbm_step(lat.ctx, -1)
    assert rc == P.lbm.LBM_EINVAL
    rc = P.lbm.lib().lbm_set_schedule(lat.ctx, 99, 0)
    assert rc == P.lbm.LBM_EINVAL

    rho0 = I.droplet_density(40, 36, 9, rl, rg)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    with pytest.raises(P.LbmError):
        lat.measure_pressure_jump(20.0, 18.0, -1.0, 14.0)
    lat.step(20)
    got = lat.read_fields(which=("rho",))["rho"]
    lat.close()
    f = O.init_equilibrium(rho0)
    O.step(op, f, 20)
    ref = O.macro(op, f)[0]
    assert np.abs(got - ref).max() <= 2e-5 * ref.max()


def test_batch_index_is_checked(P):
    eos, op, rg, rl = _cs(P)
    b = P.Batch([32, 48], [32, 40], P.LBM_FP32)
    for i in (-1, 2):
        with pytest.raises(P.LbmError) as ei:
            b.set_params(i, eos, -0.85, 0.3, rho_ref=rg)
        assert ei.value.code == P.lbm.LBM_EINVAL
    b.close()


def test_lattice_with_more_than_2_31_population_elements(P):
    """16384^2 spinodal in FP32: 9 x 16392 x 16388 = 2.4e9 elements per time
    level, so every plane offset past the first overflows 32 bits.  3 steps,
    then oracle windows (mirror-extended, as in the full-size tests) at the
    far corner, the last plane rows and seeded places, and the mass."""
    eos, op, rg, rl = _cs(P)
    n, steps, W, M = 16384, 3, 24, 6
    rho0 = I.spinodal_density(n, n, 0.25, 0.01, 14127228)
    lat = P.Lattice(n, n, P.LBM_FP32)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=0.25)
    lat.init_density(rho0)
    m0 = lat.stats()["mass"]
    lat.use_graphs(True)
    lat.step(steps)
    m1 = lat.stats()["mass"]
    rho = lat.read_fields(which=("rho",))["rho"]
    lat.close()
    assert abs(m1 / m0 - 1) < 1e-7
    rng = np.random.default_rng(16384)
    pts = [(n - 1, n - 1), (n // 2, n - 3), (n - 130, 5)] + [tuple(int(v) for v in rng.integers(0, n, 2))
                                                              for _ in range(3)]
    worst = 0.0
    for cx, cy in pts:
        ix = (np.arange(W) + cx - W // 2) % n
        iy = (np.arange(W) + cy - W // 2) % n
        w = rho0[np.ix_(iy, ix)]
        top = np.concatenate([w, w[:, ::-1]], axis=1)
        f = O.init_equilibrium(np.ascontiguousarray(np.concatenate([top, top[::-1, :]], axis=0)))
        O.step(op, f, steps)
        ref = O.macro(op, f)[0][:W, :W][M:W - M, M:W - M]
        got = rho[np.ix_(iy, ix)][M:W - M, M:W - M]
        worst = max(worst, float(np.abs(got / ref - 1).max()))
    assert worst <= 1e-6, worst


@pytest.mark.parametrize("prec", [1, 2])
def test_banded_read_back_of_a_large_lattice_matches_the_oracle_macro(P, prec):
    """A lattice of over 2^20 nodes reads its fields back in row bands (a
    band's copy to the host overlapping the next band's kernel; 1030 rows do
    not split evenly into eight): every node's rho, u and psi agree with the
    oracle's macroscopic fields of the same populations, and the initial
    state at rest is t_a rho_ref + t_a (rho - rho_ref) per population."""
    eos, op, rg, rl = _cs(P)
    nx, ny = 1040, 1030
    rho0 = I.droplet_density(nx, ny, 200, rl, rg)
    lat = P.Lattice(nx, ny, prec)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    f0 = lat.read_populations()
    rest = O.init_equilibrium(rho0)
    assert float(np.abs(f0 - rest).max() / np.abs(rest).max()) <= (1e-15 if prec == 2 else 1e-7)
    lat.step(6)
    f = lat.read_populations()
    got = lat.read_fields()
    lat.close()
    rho, ux, uy, psi = O.macro(op, f)[:4]
    assert float(np.abs(got["rho"] / rho - 1).max()) <= 1e-13
    assert float(np.abs(got["psi"] / psi - 1).max()) <= 1e-13
    assert float(np.abs(ux).max()) > 1e-6   # the drop has started to move
    assert float(np.abs(got["ux"] - ux).max()) <= 1e-14 and float(np.abs(got["uy"] - uy).max()) <= 1e-14


@pytest.mark.parametrize("prec", [1, 2])
def test_banded_initialisation_refuses_a_bad_band_and_keeps_the_state(P, prec):
    """A lattice of over 2^20 nodes takes its initial field in row bands,
    each band checked and written while the next is still being copied: a
    field with one bad value in its last band (or one bad velocity) is
    refused and leaves the populations, the step count and the steps that
    follow as they were; a good field gives, bit for bit, the populations of
    the whole-field path (which an instance of a batch takes)."""
    eos, op, rg, rl = _cs(P)
    nx, ny = 1040, 1030
    rho0 = I.droplet_density(nx, ny, 200, rl, rg)
    ux = 0.01 * np.sin(np.arange(nx * ny).reshape(ny, nx) * 0.003)
    lat = P.Lattice(nx, ny, prec)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
    lat.init_density(rho0)
    lat.step(3)
    keep = lat.read_populations()
    bad = rho0.copy()
    bad[ny - 2, 17] = np.nan
    vbad = ux.copy()
    vbad[5, 3] = np.inf
    for kw in (dict(rho=bad), dict(rho=rho0, ux=vbad)):
        with pytest.raises(P.LbmError) as ei:
            lat.init_density(**kw)
        assert ei.value.code == -1
        assert lat.steps_done == 3 and np.array_equal(lat.read_populations(), keep)
    lat.step(2)
    ref = P.Lattice(nx, ny, prec)
    ref.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
    ref.init_density(rho0)
    ref.step(5)
    assert np.array_equal(lat.read_populations(), ref.read_populations())
    ref.close()
    b = P.Batch([nx, 16], [ny, 16], prec)
    for i in range(2):
        b.set_params(i, eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
    b.init_density(1, I.droplet_density(16, 16, 4, rl, rg))
    for kw in (dict(), dict(ux=ux)):
        lat.init_density(rho0, **kw)
        b.init_density(0, rho0, **kw)
        assert lat.steps_done == 0
        assert np.array_equal(lat.read_populations(), b.read_populations(0))
    lat.step(4)
    b.step(4)
    assert np.array_equal(lat.read_populations(), b.read_populations(0))
    lat.close()
    b.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_fp32_field_interface(P, prec):
    """The FP32 entry points move half the bytes and mean the same: a float32
    initial field gives the populations of its exact float64 widening, every
    float32 field read back is the float64 one rounded to nearest (banded
    read-back of a lattice above 2^20 nodes included), and a float32 field
    is checked like a float64 one (the EOS's upper limit is excluded; NaN,
    non-positive densities and infinite velocities are refused and leave the
    state as it was)."""
    eos, op, rg, rl = _cs(P)
    for nx, ny in ((48, 40), (1040, 1030)):
        rho32 = I.droplet_density(nx, ny, min(nx, ny) / 4, rl, rg).astype(np.float32)
        ux32 = (0.01 * np.sin(np.arange(nx * ny).reshape(ny, nx) * 0.01)).astype(np.float32)
        a = P.Lattice(nx, ny, prec)
        b = P.Lattice(nx, ny, prec)
        for lat in (a, b):
            lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
        a.init_density(rho32, ux=ux32)
        b.init_density(rho32.astype(np.float64), ux=ux32.astype(np.float64))
        assert np.array_equal(a.read_populations(), b.read_populations())
        a.step(4)
        f64 = a.read_fields()
        f32 = a.read_fields(dtype=np.float32)
        for k in ("rho", "ux", "uy", "psi"):
            assert f32[k].dtype == np.float32 and np.array_equal(f32[k], f64[k].astype(np.float32)), (nx, k)
        a.close()
        b.close()
    lat = P.Lattice(48, 40, prec)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
    good = I.droplet_density(48, 40, 10, rl, rg).astype(np.float32)
    lat.init_density(good)
    lat.step(3)
    keep = lat.read_populations()
    rmax = np.float32(4.0 / 4.0)   # Carnahan-Starling: 4/b
    for field, ux in ((np.where(np.arange(48 * 40).reshape(40, 48) == 77, rmax, good), None),
                      (np.where(np.arange(48 * 40).reshape(40, 48) == 5, np.float32(np.nan), good), None),
                      (np.where(np.arange(48 * 40).reshape(40, 48) == 9, np.float32(-0.1), good), None),
                      (good, np.where(np.arange(48 * 40).reshape(40, 48) == 3, np.float32(np.inf),
                                      np.float32(0)).astype(np.float32))):
        with pytest.raises(P.LbmError) as ei:
            lat.init_density(field.astype(np.float32), ux=ux)
        assert ei.value.code == -1
        assert np.array_equal(lat.read_populations(), keep)
    just_below = np.where(np.arange(48 * 40).reshape(40, 48) == 77, np.nextafter(rmax, np.float32(0)), good)
    lat.init_density(just_below.astype(np.float32))
    lat.close()


def test_read_fields_into_caller_arrays(P):
    """read_fields fills caller-supplied (here pinned) arrays with the same
    values it returns in fresh ones, and rejects a wrong shape or dtype."""
    import torch
    eos, op, rg, rl = _cs(P)
    lat = P.Lattice(48, 40, P.LBM_FP32)
    lat.set_params(eos, -0.85, 0.3, s=S_CFG, rho_ref=rg)
    lat.init_density(I.droplet_density(48, 40, 10, rl, rg))
    lat.step(5)
    ref = lat.read_fields()
    pinned = {k: torch.empty((40, 48), dtype=torch.float64).pin_memory().numpy() for k in ("rho", "psi")}
    got = lat.read_fields(which=("rho", "psi"), out=pinned)
    assert got["rho"] is pinned["rho"] and got["psi"] is pinned["psi"]
    assert np.array_equal(got["rho"], ref["rho"]) and np.array_equal(got["psi"], ref["psi"])
    with pytest.raises(ValueError):
        lat.read_fields(which=("rho",), out={"rho": np.empty((48, 40))})
    with pytest.raises(ValueError):
        lat.read_fields(which=("rho",), out={"rho": np.empty((40, 48), dtype=np.float32)})
    lat.close()
