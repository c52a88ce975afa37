"""FP64 CPU oracle of the pseudo-potential MRT update (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  It never imports the CUDA path
and shares no code with it; the two meet only in the seeded input generators
of ``lbm_inputs``.

The stepping lives in ``lbm_oracle.c`` (plain loops, FP64); this module is the
ctypes marshalling around it plus the FP64 diagnostics of Sections 3-4 of the
paper (``oracle.analysis``).
"""
import ctypes
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None
_lib_omp = None

EOS_CS, EOS_VDW, EOS_PR = 1, 2, 3


class _Params(ctypes.Structure):
    _fields_ = [
        ("eos", ctypes.c_int),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("K", ctypes.c_double), ("T", ctypes.c_double), ("omega", ctypes.c_double),
        ("Tc", ctypes.c_double),
        ("A", ctypes.c_double), ("kappa", ctypes.c_double), ("G", ctypes.c_double),
        ("s", ctypes.c_double * 9),
        ("li_eps", ctypes.c_int), ("no_q", ctypes.c_int),
        ("fext_x", ctypes.c_double), ("fext_y", ctypes.c_double),
        ("walls_y", ctypes.c_int),
        ("var_visc", ctypes.c_int),
        ("nu_g", ctypes.c_double), ("nu_l", ctypes.c_double),
        ("visc_rho_g", ctypes.c_double), ("visc_rho_l", ctypes.c_double),
    ]


@dataclass
class Params:
    """Model parameters.  ``T`` is absolute; ``s`` is the diagonal of Lambda
    (Eq. 2) in the moment order (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy)."""
    eos: int = EOS_CS
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    K: float = 1.0
    T: float = 0.0
    omega: float = 0.0
    Tc: float = 0.0
    A: float = -0.152
    kappa: float = 0.0
    G: float = -1.0
    s: Sequence[float] = field(default_factory=lambda: [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0])
    li_eps: bool = False
    no_q: bool = False
    fext_x: float = 0.0
    fext_y: float = 0.0
    walls_y: bool = False
    var_visc: bool = False
    nu_g: float = 0.0
    nu_l: float = 0.0
    visc_rho_g: float = 0.0
    visc_rho_l: float = 1.0

    def c(self) -> _Params:
        p = _Params()
        p.eos = int(self.eos)
        for k in ("a", "b", "R", "K", "T", "omega", "Tc", "A", "kappa", "G", "fext_x", "fext_y", "nu_g", "nu_l",
                  "visc_rho_g", "visc_rho_l"):
            setattr(p, k, float(getattr(self, k)))
        p.s = (ctypes.c_double * 9)(*[float(v) for v in self.s])
        p.li_eps = int(bool(self.li_eps))
        p.no_q = int(bool(self.no_q))
        p.walls_y = int(bool(self.walls_y))
        p.var_visc = int(bool(self.var_visc))
        return p


def lib(threads: int = 1):
    """The oracle library; threads > 1 selects its OpenMP build (same bits)
    with that many threads."""
    global _lib, _lib_omp
    if threads > 1:
        if _lib_omp is None:
            _build.build()
            _lib_omp = _bind(ctypes.CDLL(_build.LIB_OMP))
        _lib_omp.orc_threads(int(threads))
        return _lib_omp
    if _lib is None:
        _build.build()
        _lib = _bind(ctypes.CDLL(_build.LIB))
    return _lib


def _bind(L):
    """Argument and result types of the oracle's C functions."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(_Params)
    L.orc_matrices.argtypes = [dp, dp]
    L.orc_velocities.argtypes = [ip, ip, dp]
    L.orc_pressure.argtypes = [pp, ctypes.c_double]
    L.orc_pressure.restype = ctypes.c_double
    L.orc_pressure_array.argtypes = [pp, dp, dp, ctypes.c_long]
    L.orc_meq.argtypes = [ctypes.c_double] * 3 + [dp]
    L.orc_source_s.argtypes = [ctypes.c_double] * 4 + [dp]
    L.orc_source_c.argtypes = [pp] + [ctypes.c_double] * 3 + [dp]
    L.orc_force_q.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp]
    L.orc_collide_node.argtypes = [pp, dp] + [ctypes.c_double] * 5 + [dp]
    L.orc_init_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
    L.orc_macro.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp]
    L.orc_macro.restype = ctypes.c_int
    L.orc_step.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
    L.orc_step.restype = ctypes.c_int
    L.orc_threads.argtypes = [ctypes.c_int]
    L.orc_threads.restype = ctypes.c_int
    return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def matrices():
    """(M, M^-1) as 9x9 float64 arrays (reading R1)."""
    M = np.zeros((9, 9))
    Mi = np.zeros((9, 9))
    lib().orc_matrices(_dp(M), _dp(Mi))
    return M, Mi


def velocities():
    ex = (ctypes.c_int * 9)()
    ey = (ctypes.c_int * 9)()
    w = np.zeros(9)
    lib().orc_velocities(ex, ey, _dp(w))
    return np.array(ex[:]), np.array(ey[:]), w


def pressure(p: Params, rho) -> np.ndarray:
    r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64))
    out = np.empty_like(r)
    pc = p.c()
    lib().orc_pressure_array(ctypes.byref(pc), _dp(r), _dp(out), r.size)
    return out


def meq(rho, vx, vy):
    out = np.zeros(9)
    lib().orc_meq(rho, vx, vy, _dp(out))
    return out


def source_s(vx, vy, Fx, Fy):
    out = np.zeros(9)
    lib().orc_source_s(vx, vy, Fx, Fy, _dp(out))
    return out


def source_c(p: Params, Qxx, Qyy, Qxy):
    out = np.zeros(9)
    pc = p.c()
    lib().orc_source_c(ctypes.byref(pc), Qxx, Qyy, Qxy, _dp(out))
    return out


def force_q(p: Params, psi: np.ndarray):
    """Eq. 9 force and Eq. 23 tensor (x G/2) from a psi field of shape (ny, nx)."""
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    ny, nx = psi.shape
    outs = [np.zeros_like(psi) for _ in range(5)]
    pc = p.c()
    lib().orc_force_q(ctypes.byref(pc), nx, ny, _dp(psi), *[_dp(o) for o in outs])
    return tuple(outs)


def collide_node(p: Params, f9, Fx, Fy, Qxx=0.0, Qyy=0.0, Qxy=0.0):
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    out = np.zeros(9)
    pc = p.c()
    lib().orc_collide_node(ctypes.byref(pc), _dp(f9), Fx, Fy, Qxx, Qyy, Qxy, _dp(out))
    return out


def init_equilibrium(rho: np.ndarray, ux: Optional[np.ndarray] = None,
                     uy: Optional[np.ndarray] = None) -> np.ndarray:
    """f = M^-1 m_eq(rho, u) with shape (9, ny, nx)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    f = np.zeros((9, ny, nx))
    uxp = _dp(np.ascontiguousarray(ux, dtype=np.float64)) if ux is not None else None
    uyp = _dp(np.ascontiguousarray(uy, dtype=np.float64)) if uy is not None else None
    lib().orc_init_equilibrium(nx, ny, _dp(rho), uxp, uyp, _dp(f))
    return f


class OracleUnstable(RuntimeError):
    pass


def step(p: Params, f: np.ndarray, n: int, threads: int = 1) -> np.ndarray:
    """Advance f (shape (9, ny, nx), modified in place) by n time steps;
    threads > 1 runs the OpenMP build (same bits)."""
    assert f.dtype == np.float64 and f.flags["C_CONTIGUOUS"] and f.shape[0] == 9
    _, ny, nx = f.shape
    pc = p.c()
    rc = lib(threads).orc_step(ctypes.byref(pc), nx, ny, _dp(f), int(n))
    if rc == 1:
        raise OracleUnstable("density left the psi domain of the EOS or became NaN")
    if rc != 0:
        raise RuntimeError("orc_step failed with %d" % rc)
    return f


def macro(p: Params, f: np.ndarray):
    """(rho, ux, uy, psi, Fx, Fy), each (ny, nx), of the current state."""
    _, ny, nx = f.shape
    outs = [np.zeros((ny, nx)) for _ in range(6)]
    pc = p.c()
    rc = lib().orc_macro(ctypes.byref(pc), nx, ny, _dp(f), *[_dp(o) for o in outs])
    if rc < 0:
        raise RuntimeError("orc_macro failed")
    return tuple(outs)


def op_count(*args) -> dict:
    """Floating-point operations of one oracle time step per lattice node,
    from the traced build of the oracle (op_count.cpp): op_count(eos, nx, ny)
    -> {flops_per_update, add_sub_per_update, mul_per_update, div_per_update,
    sqrt_per_update}; op_count("meq") or op_count("source_s") -> {flops} of
    that piece alone."""
    import subprocess
    _build.build()
    out = subprocess.run([_build.OPC_BIN] + [str(a) for a in args], check=True, capture_output=True,
                         text=True).stdout
    return {k: float(v) for k, v in (line.split("=", 1) for line in out.split())}
