"""The allocation-free entry point lbm_field_pressure_jump_static, for callers
that cannot allocate device memory: called through the C ABI on a density
field held in a device buffer, twice in a row, it must give the same Laplace
sums as lbm_batch_measure on the lattice that field came from.  This file is
collected last so a stop-at-first-failure run has run everything else; it
also passes on its own in a fresh process."""
import ctypes
import warnings

import numpy as np
import pytest

import lbm_inputs as I

warnings.filterwarnings("ignore", category=Warning, module="scipy")

pytestmark = pytest.mark.gpu

S_CFG = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]
KEYS = ("p_in", "p_out", "rho_in", "rho_out", "R_eq", "mass", "n_in", "n_out")


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_7228_gb300 as P
    P.lib()
    return P


def _eos(P, kind):
    """A law of each kind the library evaluates, below its critical point:
    Carnahan-Starling at 0.7 Tc (the droplet workloads), van der Waals at
    0.9 Tc with K = 0.3 (the paper's Table 1 case), Peng-Robinson at 0.8 Tc
    (Eq. 29 with the constants of the paper's Section 4.1)."""
    from paper_1412_7228_gb300 import experiments as X
    if kind == "cs":
        eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
        _, Tc, _ = P.lbm_eos_critical(eos)
        eos.T = 0.7 * Tc
        return eos, -0.85
    if kind == "vdw":
        return X.vdw_eos(0.9, 0.3), -0.5
    return X.pr_eos(0.8, 0.5), -0.3


def _lattice_field(P, prec, nx, ny, R, steps, kind="cs"):
    eos, A = _eos(P, kind)
    rg, rl, _ = P.lbm_eos_maxwell(eos)
    lat = P.Lattice(nx, ny, prec)
    lat.set_params(eos, A, 0.3, s=S_CFG, rho_ref=rg)
    lat.init_density(I.droplet_density(nx, ny, R, rl, rg, width=2.0 if kind == "cs" else 4.0))
    lat.step(steps)
    ref = lat.measure(0, nx / 2, ny / 2, R / 2, R + 8)
    rho = lat.read_fields(which=("rho",))["rho"]
    lat.close()
    return eos, ref, rho


def _close(got, ref, tol):
    for k in KEYS:
        assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), 1e-300), (k, got[k], ref[k])


@pytest.mark.parametrize("prec", [2, 1])
def test_static_scratch_matches_the_allocating_entry_point(P, prec):
    import torch
    stream = torch.cuda.Stream()
    # two lattices of different sizes, each sampled twice in a row, so the
    # shared scratch is reused across calls and sizes
    for nx, ny, R in ((96, 80, 18), (200, 130, 30)):
        eos, ref, rho = _lattice_field(P, prec, nx, ny, R, 150)
        d_rho = torch.from_numpy(rho).to("cuda")
        torch.cuda.synchronize()
        for _ in range(2):
            got = P.lbm.lbm_field_pressure_jump_static(d_rho.data_ptr(), nx, ny, eos, nx / 2, ny / 2, R / 2, R + 8,
                                                       stream.cuda_stream)
            _close(got, ref, 1e-12)


@pytest.mark.parametrize("kind", ["vdw", "pr"])
def test_static_scratch_matches_for_every_equation_of_state(P, kind):
    """The pressure law of the van der Waals and Peng-Robinson kinds (with
    its alpha(T) factor) gives the same sums as lbm_batch_measure."""
    import torch
    nx, ny, R = 120, 120, 30
    eos, ref, rho = _lattice_field(P, 2, nx, ny, R, 20, kind)
    d_rho = torch.from_numpy(rho).to("cuda")
    torch.cuda.synchronize()
    for _ in range(2):
        got = P.lbm.lbm_field_pressure_jump_static(d_rho.data_ptr(), nx, ny, eos, nx / 2, ny / 2, R / 2, R + 8, 0)
        _close(got, ref, 1e-12)


def test_calls_allocate_no_device_memory(P):
    """Free device memory is the same before and after calls: the entry
    point takes nothing from the device's allocator (the library and its
    static scratch were loaded by the warm-up call)."""
    import torch
    nx, ny, R = 160, 160, 30
    eos, ref, rho = _lattice_field(P, 2, nx, ny, R, 10)
    d_rho = torch.from_numpy(rho).to("cuda")
    torch.cuda.synchronize()
    P.lbm.lbm_field_pressure_jump_static(d_rho.data_ptr(), nx, ny, eos, nx / 2, ny / 2, R / 2, R + 8, 0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        got = P.lbm.lbm_field_pressure_jump_static(d_rho.data_ptr(), nx, ny, eos, nx / 2, ny / 2, R / 2, R + 8, 0)
        _close(got, ref, 1e-12)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_fields_beyond_the_static_maximum_are_rejected(P):
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.07)
    out = np.zeros(8)
    rc = P.lib().lbm_field_pressure_jump_static(ctypes.c_void_p(1 << 20), 4097, 4096, ctypes.byref(eos.c()), 1.0, 1.0,
                                                1.0, 2.0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert rc == P.lbm.LBM_EINVAL


def test_a_field_outside_device_memory_is_rejected(P):
    """A host array is refused before any GPU work (no kernel reads it)."""
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.07)
    host = np.full(64 * 64, 0.1)
    out = np.zeros(8)
    rc = P.lib().lbm_field_pressure_jump_static(host.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 64, 64,
                                                ctypes.byref(eos.c()), 32.0, 32.0, 8.0, 20.0,
                                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert rc == P.lbm.LBM_EINVAL
