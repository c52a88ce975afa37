"""Thin ctypes binding of include/lbm.h.

Argument marshalling only: every step of the method runs in the sm_103a
kernels of liblbm.so.  PyTorch supplies the device buffer handed to
lbm_create (``dev_buf``) and the CUDA stream; nothing here computes the
method.  The module fails loudly when the library has not been built.

The functions keep the C names (``lbm_create``, ``lbm_step``, ...); the
``Lattice`` and ``Batch`` classes bundle a context with its buffer and stream.
"""
import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EIO = 0, -1, -2, -3, -4, -5, -6
LBM_FP32, LBM_FP64 = 1, 2
LBM_EOS_CS, LBM_EOS_VDW, LBM_EOS_PR = 1, 2, 3
LBM_FLAG_LI_EPS = 0x1
LBM_FLAG_TEST_FORCE_TIMEOUT = 0x100
LBM_MEASURE_N = 8

_CODES = {LBM_EINVAL: "EINVAL", LBM_ENOMEM: "ENOMEM", LBM_ECUDA: "ECUDA", LBM_EUNSTABLE: "EUNSTABLE",
          LBM_ETIMEOUT: "ETIMEOUT", LBM_EIO: "EIO"}

EXPORTS = [
    "lbm_eos_pressure", "lbm_eos_critical", "lbm_eos_maxwell", "lbm_laplace_fit", "lbm_fp64_math_check",
    "lbm_fp64_fma_rate",
    "lbm_required_bytes", "lbm_batch_required_bytes", "lbm_run_chunk_plan", "lbm_create", "lbm_batch_create", "lbm_destroy",
    "lbm_set_params", "lbm_batch_set_params", "lbm_set_viscosity", "lbm_batch_set_viscosity",
    "lbm_init_density", "lbm_batch_init_density", "lbm_init_density_f32", "lbm_batch_init_density_f32",
    "lbm_step", "lbm_sync", "lbm_status", "lbm_clear_status",
    "lbm_read_fields", "lbm_batch_read_fields", "lbm_read_fields_f32", "lbm_batch_read_fields_f32",
    "lbm_read_populations", "lbm_batch_read_populations",
    "lbm_measure_pressure_jump", "lbm_batch_measure", "lbm_stats", "lbm_batch_stats",
    "lbm_save", "lbm_load", "lbm_tile_config_count", "lbm_tile_config", "lbm_set_schedule",
    "lbm_autotune", "lbm_use_graphs", "lbm_capture_graphs", "lbm_steps_done", "lbm_kernel_launches", "lbm_bytes_per_update",
    "lbm_last_error", "lbm_field_pressure_jump_static",
    "lbm_mlp_create", "lbm_mlp_destroy", "lbm_mlp_set_normalization", "lbm_mlp_set_params", "lbm_mlp_get_params",
    "lbm_mlp_loss_grad", "lbm_mlp_adam_step", "lbm_mlp_train", "lbm_mlp_predict", "lbm_mlp_invert_kappa",
]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_CODES.get(code, "?"), code, msg))
        self.code = code


class lbm_eos(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
                ("K", ctypes.c_double), ("T", ctypes.c_double), ("omega", ctypes.c_double), ("Tc", ctypes.c_double)]


@dataclass
class Eos:
    kind: int = LBM_EOS_CS
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    K: float = 1.0
    T: float = 0.0
    omega: float = 0.0
    Tc: float = 0.0

    def c(self) -> lbm_eos:
        return lbm_eos(int(self.kind), float(self.a), float(self.b), float(self.R), float(self.K), float(self.T),
                       float(self.omega), float(self.Tc))


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


def lib():
    """Load liblbm.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbm.so is not built at %s: run __graft_entry__.build() first" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    E = ctypes.POINTER(lbm_eos)
    sig = {
        "lbm_eos_pressure": ([E, ctypes.c_double, _dp], ctypes.c_int),
        "lbm_eos_critical": ([E, _dp, _dp, _dp], ctypes.c_int),
        "lbm_fp64_math_check": ([ctypes.c_double, ctypes.c_double, ctypes.c_longlong,
                                 ctypes.POINTER(ctypes.c_ulonglong)], ctypes.c_int),
        "lbm_eos_maxwell": ([E, _dp, _dp, _dp], ctypes.c_int),
        "lbm_fp64_fma_rate": ([ctypes.c_int, _vp, _dp, _dp], ctypes.c_int),
        "lbm_laplace_fit": ([ctypes.c_int, _dp, _dp, _dp, _dp, _dp], ctypes.c_int),
        "lbm_required_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
        "lbm_batch_required_bytes": ([ctypes.c_int, _ip, _ip, ctypes.c_int], ctypes.c_size_t),
        "lbm_run_chunk_plan": ([ctypes.c_int, _ip, _ip, ctypes.c_int, _ip], ctypes.c_int),
        "lbm_create": ([ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp],
                       ctypes.c_int),
        "lbm_batch_create": ([ctypes.POINTER(_vp), ctypes.c_int, _ip, _ip, ctypes.c_int, _vp, ctypes.c_size_t, _vp],
                             ctypes.c_int),
        "lbm_destroy": ([_vp], None),
        "lbm_set_params": ([_vp, E, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double,
                            ctypes.c_uint], ctypes.c_int),
        "lbm_batch_set_params": ([_vp, ctypes.c_int, E, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp,
                                  ctypes.c_double, ctypes.c_uint], ctypes.c_int),
        "lbm_set_viscosity": ([_vp, ctypes.c_int] + [ctypes.c_double] * 4, ctypes.c_int),
        "lbm_batch_set_viscosity": ([_vp, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4, ctypes.c_int),
        "lbm_init_density": ([_vp, _dp, _dp, _dp], ctypes.c_int),
        "lbm_batch_init_density": ([_vp, ctypes.c_int, _dp, _dp, _dp], ctypes.c_int),
        "lbm_init_density_f32": ([_vp, _fp, _fp, _fp], ctypes.c_int),
        "lbm_batch_init_density_f32": ([_vp, ctypes.c_int, _fp, _fp, _fp], ctypes.c_int),
        "lbm_step": ([_vp, ctypes.c_int], ctypes.c_int),
        "lbm_sync": ([_vp], ctypes.c_int),
        "lbm_status": ([_vp, ctypes.c_int], ctypes.c_int),
        "lbm_clear_status": ([_vp], ctypes.c_int),
        "lbm_read_fields": ([_vp, _dp, _dp, _dp, _dp], ctypes.c_int),
        "lbm_batch_read_fields": ([_vp, ctypes.c_int, _dp, _dp, _dp, _dp], ctypes.c_int),
        "lbm_read_fields_f32": ([_vp, _fp, _fp, _fp, _fp], ctypes.c_int),
        "lbm_batch_read_fields_f32": ([_vp, ctypes.c_int, _fp, _fp, _fp, _fp], ctypes.c_int),
        "lbm_read_populations": ([_vp, _dp], ctypes.c_int),
        "lbm_batch_read_populations": ([_vp, ctypes.c_int, _dp], ctypes.c_int),
        "lbm_measure_pressure_jump": ([_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       _dp, _dp, _dp], ctypes.c_int),
        "lbm_batch_measure": ([_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, _dp], ctypes.c_int),
        "lbm_stats": ([_vp, _dp, _dp, _dp, _dp, _dp], ctypes.c_int),
        "lbm_batch_stats": ([_vp, ctypes.c_int, _dp], ctypes.c_int),
        "lbm_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
        "lbm_load": ([_vp, ctypes.c_char_p], ctypes.c_int),
        "lbm_tile_config_count": ([ctypes.c_int], ctypes.c_int),
        "lbm_tile_config": ([ctypes.c_int, ctypes.c_int, _ip, _ip, _ip, _ip], ctypes.c_int),
        "lbm_set_schedule": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "lbm_autotune": ([_vp, ctypes.c_int, _ip, _ip, _dp], ctypes.c_int),
        "lbm_use_graphs": ([_vp, ctypes.c_int], ctypes.c_int),
        "lbm_capture_graphs": ([_vp], ctypes.c_int),
        "lbm_steps_done": ([_vp], ctypes.c_longlong),
        "lbm_kernel_launches": ([_vp], ctypes.c_longlong),
        "lbm_bytes_per_update": ([ctypes.c_int], ctypes.c_int),
        "lbm_last_error": ([_vp], ctypes.c_char_p),
        "lbm_field_pressure_jump_static": ([_vp, ctypes.c_int, ctypes.c_int, E, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, _dp, _vp], ctypes.c_int),
        "lbm_mlp_create": ([ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_ulonglong, _vp], ctypes.c_int),
        "lbm_mlp_destroy": ([_vp], None),
        "lbm_mlp_set_normalization": ([_vp, _fp, _fp, _fp, _fp], ctypes.c_int),
        "lbm_mlp_set_params": ([_vp, _fp], ctypes.c_int),
        "lbm_mlp_get_params": ([_vp, _fp], ctypes.c_int),
        "lbm_mlp_loss_grad": ([_vp, _fp, _fp, ctypes.c_int, _fp, _fp], ctypes.c_int),
        "lbm_mlp_adam_step": ([_vp, _fp, _fp, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float], ctypes.c_int),
        "lbm_mlp_train": ([_vp, _fp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                           ctypes.c_ulonglong, _fp], ctypes.c_int),
        "lbm_mlp_predict": ([_vp, _fp, ctypes.c_int, _fp], ctypes.c_int),
        "lbm_mlp_invert_kappa": ([_vp, _fp, _fp, _fp, ctypes.c_int, ctypes.c_float, ctypes.c_float, _fp],
                                 ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _ptr32(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_fp)


def _f64(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _check(ctx, rc: int):
    if rc != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        raise LbmError(rc, msg)
    return rc


# ---- host EOS helpers ----------------------------------------------------
def lbm_eos_pressure(eos: Eos, rho: float) -> float:
    p = ctypes.c_double()
    _check(None, lib().lbm_eos_pressure(ctypes.byref(eos.c()), rho, ctypes.byref(p)))
    return p.value


def lbm_eos_critical(eos: Eos):
    r, t, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(None, lib().lbm_eos_critical(ctypes.byref(eos.c()), ctypes.byref(r), ctypes.byref(t), ctypes.byref(p)))
    return r.value, t.value, p.value


def lbm_eos_maxwell(eos: Eos):
    g, l, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(None, lib().lbm_eos_maxwell(ctypes.byref(eos.c()), ctypes.byref(g), ctypes.byref(l), ctypes.byref(p)))
    return g.value, l.value, p.value


def lbm_laplace_fit(dp: Sequence[float], R: Sequence[float]):
    dp = np.ascontiguousarray(dp, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    s, c, r2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(None, lib().lbm_laplace_fit(len(dp), _ptr(dp), _ptr(R), ctypes.byref(s), ctypes.byref(c),
                                       ctypes.byref(r2)))
    return s.value, c.value, r2.value


def lbm_fp64_math_check(lo: float, hi: float, n: int) -> dict:
    """Largest distance in ulp of the FP64 step's reciprocal, division and
    square root from IEEE-rounded results over n arguments in [lo, hi], and
    whether sqrt keeps +-0 and gives NaN below zero (runs on the device)."""
    r = (ctypes.c_ulonglong * 4)()
    _check(None, lib().lbm_fp64_math_check(lo, hi, n, r))
    return {"rcp_ulp": int(r[0]), "div_ulp": int(r[1]), "sqrt_ulp": int(r[2]), "sqrt_special_ok": bool(r[3])}


def lbm_fp64_fma_rate(iters: int = 4096, stream_ptr: int = 0):
    """Measured FP64 throughput of the current device: (FLOP/s, seconds of
    the timed launch); an FMA counts as two floating-point operations."""
    f, t = ctypes.c_double(), ctypes.c_double()
    _check(None, lib().lbm_fp64_fma_rate(int(iters), ctypes.c_void_p(stream_ptr), ctypes.byref(f), ctypes.byref(t)))
    return f.value, t.value


LBM_STATIC_MAX_NODES = 16777216


def lbm_field_pressure_jump_static(d_rho_ptr: int, nx: int, ny: int, eos: Eos, cx: float, cy: float,
                                   r_in: float, r_out: float, stream_ptr: int = 0) -> dict:
    """Allocation-free Laplace sampling of a density field already in device
    memory (``d_rho_ptr``: device address of nx*ny doubles).  For callers that
    cannot allocate device memory; see include/lbm.h for the scratch rules."""
    o = np.empty(LBM_MEASURE_N)
    _check(None, lib().lbm_field_pressure_jump_static(ctypes.c_void_p(d_rho_ptr), nx, ny, ctypes.byref(eos.c()),
                                                      cx, cy, r_in, r_out, _ptr(o), ctypes.c_void_p(stream_ptr)))
    keys = ("p_in", "p_out", "rho_in", "rho_out", "R_eq", "mass", "n_in", "n_out")
    return dict(zip(keys, (float(v) for v in o)))


def lbm_required_bytes(nx: int, ny: int, precision: int) -> int:
    return int(lib().lbm_required_bytes(nx, ny, precision))


def lbm_batch_required_bytes(nx: Sequence[int], ny: Sequence[int], precision: int) -> int:
    n = len(nx)
    ax = (ctypes.c_int * n)(*nx)
    ay = (ctypes.c_int * n)(*ny)
    return int(lib().lbm_batch_required_bytes(n, ax, ay, precision))


def lbm_run_chunk_plan(nx: Sequence[int], ny: Sequence[int], precision: int) -> list:
    """The chunk (launch) of each lattice under the multi-step schedule."""
    n = len(nx)
    ax = (ctypes.c_int * n)(*nx)
    ay = (ctypes.c_int * n)(*ny)
    out = (ctypes.c_int * n)()
    rc = lib().lbm_run_chunk_plan(n, ax, ay, precision, out)
    if rc < 0:
        raise LbmError(rc, "invalid lattice shapes")
    return list(out)


def lbm_tile_configs(precision: int):
    """(tile width, tile height, threads per CTA, pipeline stages) per configuration."""
    out = []
    for k in range(lib().lbm_tile_config_count(precision)):
        bx, by, nt, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib().lbm_tile_config(precision, k, ctypes.byref(bx), ctypes.byref(by), ctypes.byref(nt), ctypes.byref(st))
        out.append((bx.value, by.value, nt.value, st.value))
    return out


DEFAULT_S = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)


class Batch:
    """A context of n independent periodic lattices stepped together
    (lbm_batch_create).  Device memory is one torch uint8 tensor; work runs
    on a dedicated torch CUDA stream unless one is given."""

    def __init__(self, nx: Sequence[int], ny: Sequence[int], precision: int = LBM_FP32, stream=None,
                 device_buffer: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        L = lib()
        self.nx = [int(v) for v in nx]
        self.ny = [int(v) for v in ny]
        self.n = len(self.nx)
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.Stream()
        nbytes = lbm_batch_required_bytes(self.nx, self.ny, precision)
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "invalid lattice shape")
        self._buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda") if device_buffer else None
        self.ctx = ctypes.c_void_p()
        ax = (ctypes.c_int * self.n)(*self.nx)
        ay = (ctypes.c_int * self.n)(*self.ny)
        buf = ctypes.c_void_p(self._buf.data_ptr()) if self._buf is not None else None
        rc = L.lbm_batch_create(ctypes.byref(self.ctx), self.n, ax, ay, precision, buf, nbytes,
                                ctypes.c_void_p(self.stream.cuda_stream))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_batch_create failed")

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().lbm_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()
        self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _c(self, rc):
        return _check(self.ctx, rc)

    def set_params(self, i: int, eos: Eos, A: float, kappa: float, G: float = -1.0, s: Sequence[float] = DEFAULT_S,
                   rho_ref: float = 0.0, flags: int = 0):
        sv = (ctypes.c_double * 9)(*[float(v) for v in s])
        self._c(lib().lbm_batch_set_params(self.ctx, i, ctypes.byref(eos.c()), A, kappa, G, sv, rho_ref, flags))

    def set_viscosity(self, i: int, nu_gas: float, nu_liquid: float, rho_gas: float, rho_liquid: float,
                      enable: bool = True):
        self._c(lib().lbm_batch_set_viscosity(self.ctx, i, int(enable), nu_gas, nu_liquid, rho_gas, rho_liquid))

    def init_density(self, i: int, rho, ux=None, uy=None):
        """Initial state of instance i from (ny, nx) fields.  float32 arrays
        (all of the given ones) go through the FP32 entry point, which moves
        half the bytes; anything else is taken as float64."""
        shape = (self.ny[i], self.nx[i])
        given = [a for a in (rho, ux, uy) if a is not None]
        if all(isinstance(a, np.ndarray) and a.dtype == np.float32 for a in given):
            r, u, v = (None if a is None else np.ascontiguousarray(a) for a in (rho, ux, uy))
            for a in (r, u, v):
                if a is not None and a.shape != shape:
                    raise ValueError("expected shape %s, got %s" % (shape, a.shape))
            self._c(lib().lbm_batch_init_density_f32(self.ctx, i, _ptr32(r), _ptr32(u), _ptr32(v)))
            return
        r, u, v = _f64(rho, shape), _f64(ux, shape), _f64(uy, shape)
        self._c(lib().lbm_batch_init_density(self.ctx, i, _ptr(r), _ptr(u), _ptr(v)))

    def step(self, n: int):
        self._c(lib().lbm_step(self.ctx, int(n)))

    def sync(self):
        self._c(lib().lbm_sync(self.ctx))

    def status(self, i: int) -> int:
        return lib().lbm_status(self.ctx, i)

    def clear_status(self):
        self._c(lib().lbm_clear_status(self.ctx))

    def read_fields(self, i: int = 0, which=("rho", "ux", "uy", "psi"), out=None, dtype=np.float64):
        """Macroscopic fields of instance i as (ny, nx) arrays of dtype
        (float64, or float32: each value rounded to nearest, half the bytes to
        move).  `out` may supply the destination arrays (e.g. in pinned
        memory, which the device-to-host copy then fills directly)."""
        dtype = np.dtype(dtype)
        if dtype not in (np.dtype(np.float64), np.dtype(np.float32)):
            raise ValueError("dtype must be float64 or float32")
        shape = (self.ny[i], self.nx[i])
        outs = {}
        for k in which:
            a = None if out is None else out.get(k)
            if a is None:
                a = np.empty(shape, dtype=dtype)
            elif a.shape != shape or a.dtype != dtype or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
                raise ValueError("out[%r] must be a writeable C-contiguous %s array of shape %s" % (k, dtype, shape))
            outs[k] = a
        keys = ("rho", "ux", "uy", "psi")
        if dtype == np.float32:
            self._c(lib().lbm_batch_read_fields_f32(self.ctx, i, *[_ptr32(outs.get(k)) for k in keys]))
        else:
            self._c(lib().lbm_batch_read_fields(self.ctx, i, *[_ptr(outs.get(k)) for k in keys]))
        return outs

    def read_populations(self, i: int = 0) -> np.ndarray:
        f = np.empty((9, self.ny[i], self.nx[i]))
        self._c(lib().lbm_batch_read_populations(self.ctx, i, _ptr(f)))
        return f

    def measure(self, i: int, cx: float, cy: float, r_in: float, r_out: float) -> dict:
        o = np.empty(LBM_MEASURE_N)
        self._c(lib().lbm_batch_measure(self.ctx, i, cx, cy, r_in, r_out, _ptr(o)))
        keys = ("p_in", "p_out", "rho_in", "rho_out", "R_eq", "mass", "n_in", "n_out")
        d = dict(zip(keys, (float(v) for v in o)))
        d["dp"] = d["p_in"] - d["p_out"]
        d["sigma"] = d["dp"] * d["R_eq"]
        return d

    def stats(self, i: int = 0) -> dict:
        o = np.empty(5)
        self._c(lib().lbm_batch_stats(self.ctx, i, _ptr(o)))
        return dict(zip(("mass", "mom_x", "mom_y", "ke", "umax"), (float(v) for v in o)))

    def save(self, path: str):
        self._c(lib().lbm_save(self.ctx, path.encode()))

    def load(self, path: str):
        self._c(lib().lbm_load(self.ctx, path.encode()))

    def set_schedule(self, tile_config: int, schedule: int = 0):
        self._c(lib().lbm_set_schedule(self.ctx, tile_config, schedule))

    def autotune(self, steps: int = 20):
        k, s, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._c(lib().lbm_autotune(self.ctx, steps, ctypes.byref(k), ctypes.byref(s), ctypes.byref(ms)))
        return k.value, s.value, ms.value

    def use_graphs(self, on: bool = True):
        self._c(lib().lbm_use_graphs(self.ctx, int(bool(on))))

    def capture_graphs(self):
        """Capture every graph step() may replay now, instead of on first use."""
        self._c(lib().lbm_capture_graphs(self.ctx))

    @property
    def steps_done(self) -> int:
        return int(lib().lbm_steps_done(self.ctx))

    @property
    def kernel_launches(self) -> int:
        return int(lib().lbm_kernel_launches(self.ctx))


class Lattice(Batch):
    """One periodic nx x ny lattice (lbm_create); instance-0 shorthands."""

    def __init__(self, nx: int, ny: int, precision: int = LBM_FP32, stream=None, device_buffer: bool = True):
        super().__init__([nx], [ny], precision, stream, device_buffer)

    def set_params(self, eos: Eos, A: float, kappa: float, G: float = -1.0, s: Sequence[float] = DEFAULT_S,
                   rho_ref: float = 0.0, flags: int = 0):
        super().set_params(0, eos, A, kappa, G, s, rho_ref, flags)

    def init_density(self, rho, ux=None, uy=None):
        super().init_density(0, rho, ux, uy)

    def measure_pressure_jump(self, cx: float, cy: float, r_in: float, r_out: float) -> dict:
        return self.measure(0, cx, cy, r_in, r_out)

    def set_viscosity(self, nu_gas: float, nu_liquid: float, rho_gas: float, rho_liquid: float,
                      enable: bool = True):
        super().set_viscosity(0, nu_gas, nu_liquid, rho_gas, rho_liquid, enable)


# ---- learned surrogate --------------------------------------------------
MLP_NPARAMS = 4676


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_fp)


class Mlp:
    """The 3-64-64-4 GELU surrogate (lbm_mlp_*): training and inference run
    in the library's CUDA kernels; this class only marshals arrays."""

    def __init__(self, max_samples: int = 4096, seed: int = 0, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.h = ctypes.c_void_p()
        _check(None, lib().lbm_mlp_create(ctypes.byref(self.h), int(max_samples), int(seed),
                                          ctypes.c_void_p(self.stream.cuda_stream)))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().lbm_mlp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        a = [_f32(v) for v in (in_mean, in_std, out_mean, out_std)]
        _check(None, lib().lbm_mlp_set_normalization(self.h, *[_fptr(v) for v in a]))

    def fit_normalization(self, X, Y):
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        self.set_normalization(X.mean(0), X.std(0) + 1e-12, Y.mean(0), Y.std(0) + 1e-12)

    def set_params(self, p):
        p = _f32(p, (MLP_NPARAMS,))
        _check(None, lib().lbm_mlp_set_params(self.h, _fptr(p)))

    def get_params(self) -> np.ndarray:
        p = np.empty(MLP_NPARAMS, dtype=np.float32)
        _check(None, lib().lbm_mlp_get_params(self.h, _fptr(p)))
        return p

    def loss_grad(self, X, Y):
        X = _f32(X)
        Y = _f32(Y)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(MLP_NPARAMS, dtype=np.float32)
        _check(None, lib().lbm_mlp_loss_grad(self.h, _fptr(X), _fptr(Y), len(X), _fptr(loss), _fptr(g)))
        return float(loss[0]), g

    def adam_step(self, X, Y, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        X = _f32(X)
        Y = _f32(Y)
        _check(None, lib().lbm_mlp_adam_step(self.h, _fptr(X), _fptr(Y), len(X), lr, beta1, beta2, eps))

    def train(self, X, Y, epochs=200, batch=128, lr=1e-3, seed=0):
        X = _f32(X)
        Y = _f32(Y)
        losses = np.zeros(epochs, dtype=np.float32)
        _check(None, lib().lbm_mlp_train(self.h, _fptr(X), _fptr(Y), len(X), epochs, batch, lr, seed,
                                         _fptr(losses)))
        return losses

    def predict(self, X) -> np.ndarray:
        X = _f32(X)
        Y = np.empty((len(X), 4), dtype=np.float32)
        _check(None, lib().lbm_mlp_predict(self.h, _fptr(X), len(X), _fptr(Y)))
        return Y

    def invert_kappa(self, t_over_tc, A, sigma, lo=0.0, hi=0.6) -> np.ndarray:
        t = _f32(t_over_tc)
        a = _f32(A)
        s = _f32(sigma)
        k = np.empty(len(t), dtype=np.float32)
        _check(None, lib().lbm_mlp_invert_kappa(self.h, _fptr(t), _fptr(a), _fptr(s), len(t), lo, hi, _fptr(k)))
        return k
