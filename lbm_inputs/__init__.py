"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method: only the
initial density fields of the paper's workloads (static droplet, flat
interface, spinodal noise) and the seeded parameter draws of the batched
sweep.  Coexistence densities are passed in by the caller; nothing here
evaluates an equation of state.

Random numbers: the spinodal noise uses splitmix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) keyed by
``seed ^ node_index``, so any side can regenerate any node; parameter draws use
numpy's PCG64 (``numpy.random.default_rng``), identical on every platform.
"""
from dataclasses import dataclass
from typing import List

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64 finaliser over uint64 keys."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """u in [-1, 1) for node indices 0..n-1: top 53 bits of splitmix64(seed ^ i)."""
    idx = np.arange(n, dtype=np.uint64)
    z = splitmix64(np.uint64(seed) ^ idx)
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u01 - 1.0


def spinodal_density(nx: int, ny: int, rho0: float = 0.25, amp: float = 0.01,
                     seed: int = 14127228) -> np.ndarray:
    """Uniform density with seeded +-amp relative noise: rho0 (1 + amp u)."""
    u = uniform_pm1(seed, nx * ny).reshape(ny, nx)
    return rho0 * (1.0 + amp * u)


def _min_image(nx: int, ny: int, cx: float, cy: float) -> np.ndarray:
    dx = np.arange(nx, dtype=np.float64)[None, :] - cx
    dy = np.arange(ny, dtype=np.float64)[:, None] - cy
    dx = dx - nx * np.round(dx / nx)
    dy = dy - ny * np.round(dy / ny)
    return np.sqrt(dx * dx + dy * dy)


def droplet_density(nx: int, ny: int, radius: float, rho_l: float, rho_g: float,
                    width: float = 2.0, cx: float = None, cy: float = None) -> np.ndarray:
    """Static droplet: rho_g + (rho_l - rho_g)/2 * (1 - tanh(2 (r - R) / W)),
    centred at (nx/2, ny/2) unless given, r the periodic minimum-image distance
    from node coordinates."""
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    r = _min_image(nx, ny, cx, cy)
    return rho_g + 0.5 * (rho_l - rho_g) * (1.0 - np.tanh(2.0 * (r - radius) / width))


def slab_density(nx: int, ny: int, rho_l: float, rho_g: float, width: float = 2.0) -> np.ndarray:
    """Flat interfaces normal to x, liquid in the centre half [nx/4, 3nx/4)."""
    x = np.arange(nx, dtype=np.float64)
    x1, x2 = nx / 4.0, 3.0 * nx / 4.0
    prof = rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (x - x1) / width)
                                            - np.tanh(2.0 * (x - x2) / width))
    return np.broadcast_to(prof[None, :], (ny, nx)).copy()


def ellipse_density(nx: int, ny: int, r_major: float, r_minor: float, rho_l: float,
                    rho_g: float, width: float = 2.0) -> np.ndarray:
    """Elliptic drop (major axis along x) for the oscillation experiment."""
    dx = np.arange(nx, dtype=np.float64)[None, :] - nx / 2.0
    dy = np.arange(ny, dtype=np.float64)[:, None] - ny / 2.0
    s = np.sqrt((dx / r_major) ** 2 + (dy / r_minor) ** 2)
    r_eff = np.sqrt(r_major * r_minor)
    return rho_g + 0.5 * (rho_l - rho_g) * (1.0 - np.tanh(2.0 * (s - 1.0) * r_eff / width))


@dataclass
class SweepInstance:
    L: int            # square domain edge
    radius: float     # droplet radius, 0.2 L
    T_over_Tc: float
    A: float
    kappa: float


def sweep_instances(n: int = 64, seed: int = 7228, sizes=(128, 256, 512, 1024)) -> List[SweepInstance]:
    """Batched uneven sweep: L uniform over ``sizes``, R = 0.2 L,
    T/Tc ~ U[0.6, 0.85], A ~ U[-0.2, -0.1], kappa ~ U[0, 0.6]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = int(sizes[int(rng.integers(0, len(sizes)))])
        t = float(rng.uniform(0.6, 0.85))
        A = float(rng.uniform(-0.2, -0.1))
        k = float(rng.uniform(0.0, 0.6))
        out.append(SweepInstance(L=L, radius=0.2 * L, T_over_Tc=t, A=A, kappa=k))
    return out
