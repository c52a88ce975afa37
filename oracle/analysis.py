"""FP64 diagnostics of the paper's experiments (TEST INFRASTRUCTURE).

Equations of state with their analytic derivatives, the critical point, the
Maxwell equal-area coexistence, the mechanical-stability coexistence of Eq. 17,
and the field diagnostics of Sections 3-4: Laplace's law (Eq. 22), the
equimolar droplet radius, flat-interface densities (Table 1) and the
flat-interface surface tension of Eq. 20.  numpy/scipy only; nothing here is
shared with the CUDA path.
"""
import math
from typing import Optional, Tuple

import numpy as np
from scipy import integrate, optimize

from . import EOS_CS, EOS_PR, EOS_VDW, Params


# --------------------------------------------------------------------------
# Equations of state (K scales the whole law, reading R8)
# --------------------------------------------------------------------------
def p_eos(p: Params, rho):
    """Pressure: Carnahan-Starling, van der Waals (Eq. 21), Peng-Robinson (Eq. 29)."""
    rho = np.asarray(rho, dtype=np.float64)
    RT = p.R * p.T
    if p.eos == EOS_CS:
        eta = p.b * rho / 4.0
        return p.K * (rho * RT * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - p.a * rho**2)
    if p.eos == EOS_VDW:
        return p.K * (rho * RT / (1 - p.b * rho) - p.a * rho**2)
    if p.eos == EOS_PR:
        alpha = pr_alpha(p)
        br = p.b * rho
        return p.K * (rho * RT / (1 - br) - p.a * alpha * rho**2 / (1 + 2 * br - br**2))
    raise ValueError("unknown EOS")


def pr_alpha(p: Params) -> float:
    """alpha(T) of Eq. 29."""
    m = 0.37464 + 1.54226 * p.omega - 0.26992 * p.omega**2
    return (1 + m * (1 - math.sqrt(p.T / p.Tc))) ** 2


def dp_drho(p: Params, rho):
    """Analytic dp/drho of the three laws."""
    rho = np.asarray(rho, dtype=np.float64)
    RT = p.R * p.T
    if p.eos == EOS_CS:
        eta = p.b * rho / 4.0
        return p.K * (RT * (1 + 4 * eta + 4 * eta**2 - 4 * eta**3 + eta**4) / (1 - eta) ** 4
                      - 2 * p.a * rho)
    if p.eos == EOS_VDW:
        return p.K * (RT / (1 - p.b * rho) ** 2 - 2 * p.a * rho)
    if p.eos == EOS_PR:
        alpha = pr_alpha(p)
        br = p.b * rho
        D = 1 + 2 * br - br**2
        return p.K * (RT / (1 - br) ** 2 - p.a * alpha * (2 * rho + 2 * p.b * rho**2) / D**2)
    raise ValueError("unknown EOS")


def rho_max(p: Params) -> float:
    """Upper end of the EOS's physical density range (pole or packing limit)."""
    if p.eos == EOS_CS:
        return 4.0 / p.b
    return 1.0 / p.b


def with_T(p: Params, T: float) -> Params:
    q = Params(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.T = T
    return q


def critical_point(p: Params) -> Tuple[float, float, float]:
    """(rho_c, T_c, p_c): the temperature at which the minimum over rho of
    dp/drho reaches zero; rho_c is where that minimum sits."""
    hi = rho_max(p)

    def min_slope(T):
        q = with_T(p, T)
        r = optimize.minimize_scalar(lambda x: float(dp_drho(q, x)), bounds=(1e-9 * hi, 0.999 * hi),
                                     method="bounded", options={"xatol": 1e-14 * hi, "maxiter": 2000})
        return r.fun, r.x

    # bracket T_c: at very low T the slope goes negative, at high T it is positive
    T_lo, T_hi = 1e-6, 1.0
    while min_slope(T_hi)[0] <= 0:
        T_hi *= 2
    Tc = optimize.brentq(lambda T: min_slope(T)[0], T_lo, T_hi, xtol=1e-15, rtol=1e-14, maxiter=500)
    _, rc = min_slope(Tc)
    pc = float(p_eos(with_T(p, Tc), rc))
    return float(rc), float(Tc), pc


def spinodal(p: Params) -> Tuple[float, float]:
    """The two densities where dp/drho = 0 (below T_c)."""
    hi = rho_max(p)
    r = optimize.minimize_scalar(lambda x: float(dp_drho(p, x)), bounds=(1e-9 * hi, 0.999 * hi),
                                 method="bounded", options={"xatol": 1e-14 * hi, "maxiter": 2000})
    if r.fun >= 0:
        raise ValueError("temperature is not below the critical temperature")
    rm = r.x
    s1 = optimize.brentq(lambda x: float(dp_drho(p, x)), 1e-12 * hi, rm, xtol=1e-16)
    s2 = optimize.brentq(lambda x: float(dp_drho(p, x)), rm, 0.99999 * hi, xtol=1e-16)
    return s1, s2


def _roots_at(p: Params, p0: float, s1: float, s2: float) -> Tuple[float, float]:
    hi = rho_max(p)
    rg = optimize.brentq(lambda x: float(p_eos(p, x)) - p0, 1e-300, s1, xtol=1e-300, rtol=1e-15)
    top = 0.99999999 * hi
    rl = optimize.brentq(lambda x: float(p_eos(p, x)) - p0, s2, top, xtol=1e-16, rtol=1e-15)
    return rg, rl


def _quad(fn, lo, hi):
    """int_lo^hi fn with scipy's adaptive Gauss-Kronrod: (value, error estimate).
    full_output keeps scipy from warning; the caller judges the estimate."""
    val, err, *_ = integrate.quad(fn, lo, hi, limit=400, epsabs=1e-16, epsrel=1e-13, full_output=1)
    return val, err


def _coexistence(p: Params, weight) -> Optional[Tuple[float, float, float]]:
    """Solve p(rho_g) = p(rho_l) = p0 and int_{rho_g}^{rho_l} (p0 - p) weight drho = 0.

    The integral is split at the spinodal densities s1 < s2, where p has its
    turning points, into the gas, unstable and liquid branches.  The gas
    branch runs over rho_g .. s1 with rho_g as small as p0 allows, so it is
    integrated in u = ln rho (drho = rho du), which spreads its decades
    evenly; the weight of Eq. 17 grows like a power of 1/rho there.  The
    coexistence pressure is returned only when the summed error estimate at
    the root is below 1e-9 of the largest branch integral."""
    s1, s2 = spinodal(p)
    p_hi = float(p_eos(p, s1))
    p_lo = max(float(p_eos(p, s2)), 0.0)
    eps = 1e-13 * max(abs(p_hi), 1e-300)

    def f(p0, x):
        return (p0 - float(p_eos(p, x))) * weight(x)

    def F(p0, full=False):
        rg, rl = _roots_at(p, p0, s1, s2)
        gas = _quad(lambda u: f(p0, math.exp(u)) * math.exp(u), math.log(rg), math.log(s1))
        mid = _quad(lambda x: f(p0, x), s1, s2)
        liq = _quad(lambda x: f(p0, x), s2, rl)
        val = gas[0] + mid[0] + liq[0]
        if full:
            return val, gas[1] + mid[1] + liq[1], max(abs(gas[0]), abs(mid[0]), abs(liq[0]))
        return val

    a, b = p_lo + eps, p_hi - eps
    fa, fb = F(a), F(b)
    if not (fa * fb < 0):
        return None
    p0 = optimize.brentq(F, a, b, xtol=1e-18, rtol=1e-14, maxiter=500)
    _, err, scale = F(p0, full=True)
    if not err <= 1e-9 * scale:
        raise ArithmeticError("coexistence integral not resolved: error estimate %.3g of %.3g" % (err, scale))
    rg, rl = _roots_at(p, p0, s1, s2)
    return rg, rl, p0


def maxwell(p: Params) -> Tuple[float, float, float]:
    """Thermodynamic coexistence (Maxwell equal area in 1/rho): (rho_g, rho_l, p0)."""
    r = _coexistence(p, lambda x: 1.0 / (x * x))
    if r is None:
        raise ValueError("no Maxwell coexistence found")
    return r


def psi_of_rho(p: Params, rho):
    """Eq. 10 with c = 1 (R7): psi = sqrt(2 (p_EOS - rho/3) / G)."""
    return np.sqrt(2.0 * (p_eos(p, rho) - np.asarray(rho) / 3.0) / p.G)


def dpsi_drho(p: Params, rho):
    """From psi^2 = 2 (p - rho/3) / G:  psi' = (p' - 1/3) / (G psi)."""
    return (dp_drho(p, rho) - 1.0 / 3.0) / (p.G * psi_of_rho(p, rho))


def mechanical_stability(p: Params, eps: Optional[float] = None):
    """Coexistence densities from the mechanical-stability condition Eq. 17,
    int (p0 - p_EOS) psi' / psi^(1+eps) drho = 0, with eps = -2a/b and the
    a = 3A, b = 3 of Eqs. 14-15, i.e. eps = -2A (reading R9).  Returns
    (rho_g, rho_l, p0) or None when no solution with p0 > 0 exists."""
    if eps is None:
        eps = -2.0 * p.A
    return _coexistence(p, lambda x: float(dpsi_drho(p, x) / psi_of_rho(p, x) ** (1.0 + eps)))


# --------------------------------------------------------------------------
# Field diagnostics
# --------------------------------------------------------------------------
def min_image_radius(nx: int, ny: int, cx: float, cy: float) -> np.ndarray:
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    dx = x[None, :] - cx
    dy = y[:, None] - cy
    dx = dx - nx * np.round(dx / nx)
    dy = dy - ny * np.round(dy / ny)
    return np.sqrt(dx * dx + dy * dy)


def pressure_jump(p: Params, rho: np.ndarray, cx: float, cy: float, r_in: float, r_out: float):
    """Laplace-law sampling (Eq. 22): mean pressure p = rho/3 + G psi^2/2 =
    p_EOS(rho) (Eq. 10) over r <= r_in and over r >= r_out (minimum image), the
    mean densities there, and the equimolar radius
    R_eq = sqrt((sum rho - rho_out N) / (pi (rho_in - rho_out)))."""
    ny, nx = rho.shape
    r = min_image_radius(nx, ny, cx, cy)
    pf = p_eos(p, rho)
    inside = r <= r_in
    outside = r >= r_out
    p_in = float(pf[inside].mean())
    p_out = float(pf[outside].mean())
    rho_in = float(rho[inside].mean())
    rho_out = float(rho[outside].mean())
    mass = float(rho.sum())
    R_eq = math.sqrt(max(mass - rho_out * nx * ny, 0.0) / (math.pi * (rho_in - rho_out)))
    return dict(p_in=p_in, p_out=p_out, dp=p_in - p_out, rho_in=rho_in, rho_out=rho_out,
                R_eq=R_eq, mass=mass, sigma=(p_in - p_out) * R_eq)


def laplace_fit(dp, R):
    """Least-squares line dp = sigma * (1/R) + c (Eq. 22): (sigma, c, r^2)."""
    x = 1.0 / np.asarray(R, dtype=np.float64)
    y = np.asarray(dp, dtype=np.float64)
    X = np.stack([x, np.ones_like(x)], axis=1)
    (slope, icpt), *_ = np.linalg.lstsq(X, y, rcond=None)
    yhat = X @ np.array([slope, icpt])
    ss_res = float(((y - yhat) ** 2).sum())
    ss_tot = float(((y - y.mean()) ** 2).sum())
    r2 = 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0
    return float(slope), float(icpt), r2


def slab_densities(rho: np.ndarray) -> Tuple[float, float]:
    """Flat interface along x with the liquid in the centre half: rho_l at the
    centre column, rho_g at the column furthest from it (the domain edge)."""
    prof = rho.mean(axis=0)
    nx = prof.size
    return float(prof[nx // 2]), float(prof[0])


def sigma_flat_eq20(p: Params, rho_profile: np.ndarray) -> float:
    """Eq. 20 with the kappa factor of Eq. 28, summed over both interfaces of a
    periodic slab and halved: sigma = (1 - kappa) (A - 1) (G/6) int psi'^2 dn,
    with central differences for psi'."""
    psi = psi_of_rho(p, rho_profile)
    d = 0.5 * (np.roll(psi, -1) - np.roll(psi, 1))
    return 0.5 * (1.0 - p.kappa) * (p.A - 1.0) * (p.G / 6.0) * float((d * d).sum())
