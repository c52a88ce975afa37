"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/lbm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def liblbm():
    from paper_1412_7228_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_function_is_exported(liblbm):
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(liblbm, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1412_7228_gb300 import lbm
    assert sorted(lbm.EXPORTS) == declared_functions()


def test_host_only_calls_work_without_a_gpu(liblbm):
    import paper_1412_7228_gb300 as P
    assert P.lbm_required_bytes(64, 64, P.LBM_FP32) > 0
    assert P.lbm_required_bytes(1, 64, P.LBM_FP32) == 0          # nx < 2 is rejected
    assert P.lbm_required_bytes(64, 64, 3) == 0                  # unknown precision
    assert liblbm.lbm_bytes_per_update(P.LBM_FP32) == 72
    assert liblbm.lbm_bytes_per_update(P.LBM_FP64) == 144
    cfgs = P.lbm_tile_configs(P.LBM_FP32)
    assert (128, 16, 512, 1) in cfgs and all(c[3] in (1, 2) for c in cfgs)


def test_product_eos_helpers_agree_with_the_oracle():
    """The library's own critical-point and Maxwell solvers (host C++) against
    the oracle's independent scipy ones."""
    import warnings
    warnings.filterwarnings("ignore")
    import oracle as O
    from oracle import analysis as An
    import paper_1412_7228_gb300 as P
    e = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    rc, Tc, pc = P.lbm_eos_critical(e)
    orc = An.critical_point(O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0))
    assert abs(Tc / orc[1] - 1) < 1e-10 and abs(rc / orc[0] - 1) < 1e-6
    for tr in (0.6, 0.7, 0.8):
        e.T = tr * Tc
        g, l, p0 = P.lbm_eos_maxwell(e)
        og, ol, op0 = An.maxwell(An.with_T(O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0), tr * orc[1]))
        assert abs(g / og - 1) < 1e-8 and abs(l / ol - 1) < 1e-8
    for rho in (0.01, 0.2, 0.4):
        ref = O.pressure(An.with_T(O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0), e.T), [rho])[0]
        assert abs(P.lbm_eos_pressure(e, rho) - ref) < 1e-15
    s, c, r2 = P.lbm_laplace_fit([0.3, 0.2, 0.15], [10.0, 15.0, 20.0])
    assert abs(s - 3.0) < 1e-12 and abs(c) < 1e-12 and abs(r2 - 1) < 1e-12


@pytest.mark.parametrize("bad", [dict(T=0.0), dict(T=-0.07), dict(T=float("nan")), dict(a=0.0), dict(b=-4.0),
                                 dict(R=0.0), dict(K=0.0), dict(kind=7), dict(kind=3, Tc=0.0)])
def test_static_sampling_rejects_what_set_params_rejects(liblbm, bad):
    """lbm_field_pressure_jump_static refuses an equation of state or a
    temperature that lbm_set_params refuses, before it touches the GPU
    (the pointer is never dereferenced: no GPU is needed here)."""
    import numpy as np
    import paper_1412_7228_gb300 as P
    kw = dict(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, T=0.07, omega=0.344, Tc=0.1)
    kw.update(bad)
    eos = P.Eos(**kw)
    out = np.zeros(8)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = P.lib().lbm_field_pressure_jump_static(ctypes.c_void_p(1 << 20), 64, 64, ctypes.byref(eos.c()), 32.0, 32.0,
                                                8.0, 20.0, out.ctypes.data_as(dp), None)
    assert rc == P.lbm.LBM_EINVAL
    assert P.lib().lbm_eos_maxwell(ctypes.byref(eos.c()), out.ctypes.data_as(dp), out.ctypes.data_as(dp),
                                   out.ctypes.data_as(dp)) == P.lbm.LBM_EINVAL


def test_context_calls_refuse_a_null_context(liblbm):
    """Every call that takes a context returns LBM_EINVAL for NULL, before any
    GPU work (so these run without a GPU)."""
    import paper_1412_7228_gb300 as P
    L = P.lib()
    E = P.lbm.LBM_EINVAL
    assert L.lbm_step(None, 1) == E
    assert L.lbm_set_schedule(None, 0, 4) == E
    assert L.lbm_use_graphs(None, 1) == E
    assert L.lbm_capture_graphs(None) == E
    assert L.lbm_init_density(None, None, None, None) == E
    assert L.lbm_init_density_f32(None, None, None, None) == E
    assert L.lbm_read_fields(None, None, None, None, None) == E
    assert L.lbm_read_fields_f32(None, None, None, None, None) == E
    assert L.lbm_batch_init_density_f32(None, 0, None, None, None) == E
    assert L.lbm_batch_read_fields_f32(None, 0, None, None, None, None) == E


C_PROGRAM = r"""
#include <stdio.h>
#include "lbm.h"

int main(void) {
    lbm_eos eos = {LBM_EOS_CS, 1.0, 4.0, 1.0, 1.0, 0.0, 0.0, 0.0};
    double rho_c, T_c, p_c;
    int nx[3] = {256, 256, 4096}, ny[3] = {256, 256, 4096}, chunk_of[3];
    int bx, by, threads, stages, chunks;
    if (lbm_eos_critical(&eos, &rho_c, &T_c, &p_c) != LBM_OK) return 1;
    if (lbm_tile_config(LBM_FP32, 0, &bx, &by, &threads, &stages) != LBM_OK) return 2;
    chunks = lbm_run_chunk_plan(3, nx, ny, LBM_FP32, chunk_of);
    printf("%.9f %.9f %d %d %d %d %d %zu %d %d %d %d\n", rho_c, T_c, bx, by, threads, stages,
           lbm_bytes_per_update(LBM_FP32), lbm_required_bytes(1, 64, LBM_FP32), chunks, chunk_of[0],
           chunk_of[1], chunk_of[2]);
    return 0;
}
"""


def test_header_is_plain_c_and_host_calls_link_from_c(liblbm, tmp_path):
    """include/lbm.h compiles as strict C99 (no C++ in the boundary), and a C
    program links against liblbm.so and makes the host-only calls."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_lbm.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_lbm"
    lib_dir = os.path.dirname(liblbm._name)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", lib_dir, "-llbm", "-Wl,-rpath," + lib_dir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    v = out.stdout.split()
    assert abs(float(v[0]) - 0.130444) < 1e-5 and abs(float(v[1]) - 0.0943287) < 1e-6   # R15
    assert v[2:6] == ["128", "16", "512", "1"] and v[6] == "72"
    assert v[7] == "0"                                     # nx = 1 is refused
    assert v[8:] == ["2", "1", "1", "0"]                    # the 4096^2 lattice alone, first


def test_laplace_fit_agrees_with_the_oracle_and_refuses_degenerate_input(liblbm):
    """The library's FP64 least squares of Eq. 22 against the oracle's on
    noisy points; fewer than two points, a non-positive radius or a single
    radius (no slope) are refused."""
    import numpy as np
    from oracle import analysis as An
    import paper_1412_7228_gb300 as P
    rng = np.random.default_rng(5)
    R = np.array([16.1, 28.1, 38.8, 49.3, 59.6])
    dp = 0.012 / R + 7e-6 + rng.normal(0.0, 2e-6, R.size)
    s, c, r2 = P.lbm_laplace_fit(list(dp), list(R))
    so, co, r2o = An.laplace_fit(list(dp), list(R))
    assert abs(s / so - 1) < 1e-12 and abs(c - co) < 1e-15 and abs(r2 - r2o) < 1e-12 and 0.99 < r2 < 1
    for dps, Rs in (([1e-3], [10.0]), ([1e-3, 2e-3], [10.0, 0.0]), ([1e-3, 2e-3], [10.0, -5.0]),
                    ([1e-3, 2e-3, 3e-3], [12.0, 12.0, 12.0])):
        with pytest.raises(P.LbmError):
            P.lbm_laplace_fit(dps, Rs)
