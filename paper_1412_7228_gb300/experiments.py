"""The paper's other experiments, run on the GPU path.

- ``method1``: surface tension against the hybrid weight A (Section 3.1.1,
  Fig. 1) from R = 20 droplets in 100x100, and the flat-interface
  densities against A (Section 3.1.2, Fig. 2), van der Waals law
  (a = 9/49, b = 2/21, R = 1, K = 0.3, T = 0.9 Tc).
- ``pr_laplace``: Laplace's law with the Peng-Robinson law (Section 4.1,
  Fig. 4): 120x120, radii 20-40, kappa in {0, 0.9, 0.99}, T = 0.8 Tc,
  A = -0.3, K = 0.5, omega = 0.344, b = 2/21, R = 1.  The paper does not
  print a; PR_A is the a for which the simulated flat interface has the
  density ratio of 430 it states.  The same a gives, without further
  tuning, an interface 3.6 nodes wide (the paper: about 4) and sigma = 0.161
  at kappa = 0 (the paper's Section 4.2 uses 0.16).  With the customary
  a = 2/49 the flat interface diverges at these parameters.
- ``oscillation``: an elliptic cylinder (30 x 27) relaxing to a circle in
  120x120 (Section 4.2) with the gas/liquid viscosities of the paper; the
  period against T = 2 pi sqrt(rho_l R0^3 / (n (n^2 - 1) sigma)), n = 2,
  R0 = sqrt(30 27) (Eq. 30, read with 2 pi outside the root, which is the
  form that reproduces the theory periods the paper prints).

Host orchestration over the C ABI; every lattice update runs in liblbm.so.
``python -m paper_1412_7228_gb300.experiments --help``.
"""
import argparse
import json
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

import lbm_inputs as I

from . import lbm as L

S_ONES = (1.0,) * 9
PR_A = 0.0703
PR_B = 2.0 / 21.0
PR_OMEGA = 0.344


def vdw_eos(t_over_tc: float = 0.9, K: float = 0.3) -> L.Eos:
    eos = L.Eos(kind=L.LBM_EOS_VDW, a=9.0 / 49.0, b=2.0 / 21.0, R=1.0, K=K)
    _, Tc, _ = L.lbm_eos_critical(eos)
    eos.T = t_over_tc * Tc
    return eos


def pr_eos(t_over_tc: float = 0.8, K: float = 0.5, a: float = PR_A) -> L.Eos:
    """Peng-Robinson law (Eq. 29) with b = 2/21, R = 1, omega = 0.344 and
    Tc = 0.0778 a / (0.45724 b R), the critical temperature those constants fix."""
    Tc = 0.0778 * a / (0.45724 * PR_B)
    return L.Eos(kind=L.LBM_EOS_PR, a=a, b=PR_B, R=1.0, K=K, T=t_over_tc * Tc, omega=PR_OMEGA, Tc=Tc)


def slabs(eos: L.Eos, cases: Sequence[Tuple[float, float]], rho_l0: float, rho_g0: float, steps: int = 20000,
          nx: int = 128, ny: int = 4, s=S_ONES, precision: int = L.LBM_FP64) -> List[Tuple[float, float]]:
    """Flat interfaces (liquid in the centre half) for each (A, kappa):
    returns (rho_l at the centre column, rho_g at the domain edge)."""
    b = L.Batch([nx] * len(cases), [ny] * len(cases), precision)
    rho0 = I.slab_density(nx, ny, rho_l0, rho_g0, width=4.0)
    for i, (A, k) in enumerate(cases):
        b.set_params(i, eos, A, k, G=-1.0, s=s, rho_ref=rho_g0)
        b.init_density(i, rho0)
    b.use_graphs(True)
    b.autotune(40)   # tile and schedule: the same bits in every one
    b.step(steps)
    out = []
    for i in range(len(cases)):
        prof = b.read_fields(i, which=("rho",))["rho"].mean(axis=0)
        out.append((float(prof[nx // 2]), float(prof[0])))
    b.close()
    return out


def droplets(eos: L.Eos, cases: Sequence[Tuple[float, float, float]], L_: int, rho_l0: float, rho_g0: float,
             steps: int, s=S_ONES, precision: int = L.LBM_FP32, gap: float = 10.0, width: float = 4.0) -> List[Dict]:
    """Static droplets (A, kappa, R0) at the centre of L_ x L_: Laplace
    sampling (Eq. 22) after `steps` steps."""
    b = L.Batch([L_] * len(cases), [L_] * len(cases), precision)
    for i, (A, k, R) in enumerate(cases):
        b.set_params(i, eos, A, k, G=-1.0, s=s, rho_ref=rho_g0)
        b.init_density(i, I.droplet_density(L_, L_, R, rho_l0, rho_g0, width=width))
    b.use_graphs(True)
    b.autotune(40)
    b.step(steps)
    out = []
    for i, (A, k, R) in enumerate(cases):
        st = b.status(i)
        m = b.measure(i, L_ / 2.0, L_ / 2.0, R / 2.0, R + gap) if st == 0 else {}
        m.update(A=A, kappa=k, R0=R, status=st)
        out.append(m)
    b.clear_status()
    b.close()
    return out


def method1(As=(-0.9, -0.5, 0.0, 0.5, 0.9, 0.99), steps_drop: int = 6000, steps_slab: int = 20000) -> Dict:
    """Fig. 1 (sigma vs A, kappa = 0) and Fig. 2 (rho_l, rho_g vs A)."""
    eos = vdw_eos()
    drops = droplets(eos, [(A, 0.0, 20.0) for A in As], 100, 5.79198, 1.46621, steps_drop)
    sl = slabs(eos, [(A, 0.0) for A in As], 5.8, 1.47, steps_slab)
    return {"A": list(As), "sigma": [d.get("sigma", float("nan")) for d in drops],
            "rho_l": [v[0] for v in sl], "rho_g": [v[1] for v in sl]}


def pr_coexistence(kappa: float = 0.0, A: float = -0.3, steps: int = 30000) -> Tuple[float, float]:
    eos = pr_eos()
    return slabs(eos, [(A, kappa)], 7.17, 0.0167, steps)[0]


def interface_width(profile: np.ndarray) -> float:
    """10-90 % width of the left interface of a slab profile (liquid in the
    centre half), in lattice units."""
    n = profile.size
    lo, hi = profile[0], profile[n // 2]
    z = (profile[: n // 2] - lo) / (hi - lo)
    x = np.arange(n // 2, dtype=np.float64)
    return float(np.interp(0.9, z, x) - np.interp(0.1, z, x))


def pr_laplace(kappas=(0.0, 0.9, 0.99), radii=(20, 25, 30, 35, 40), L_: int = 120, steps: int = 20000,
               A: float = -0.3, precision: int = L.LBM_FP32) -> Dict:
    eos = pr_eos()
    rl, rg = pr_coexistence(0.0, A)
    res = droplets(eos, [(A, k, float(R)) for k in kappas for R in radii], L_, rl, rg, steps, precision=precision)
    fits = {}
    for k in kappas:
        grp = [d for d in res if d["kappa"] == k and d["status"] == 0 and d["R_eq"] >= 0.75 * d["R0"]]
        if len(grp) >= 2:
            sigma, icpt, r2 = L.lbm_laplace_fit([d["dp"] for d in grp], [d["R_eq"] for d in grp])
            fits[k] = {"sigma": sigma, "intercept": icpt, "r2": r2, "dp": [d["dp"] for d in grp],
                       "R_eq": [d["R_eq"] for d in grp], "rho_in": [d["rho_in"] for d in grp],
                       "rho_out": [d["rho_out"] for d in grp]}
    return {"rho_l": rl, "rho_g": rg, "ratio": rl / rg, "fits": fits}


def deformation(rho: np.ndarray, rho_g: float) -> float:
    """Second-moment anisotropy sum (rho - rho_g)(dx^2 - dy^2) about the centre."""
    ny, nx = rho.shape
    dx = np.arange(nx)[None, :] - nx / 2.0
    dy = np.arange(ny)[:, None] - ny / 2.0
    w = rho - rho_g
    return float((w * (dx * dx - dy * dy)).sum() / w.sum())


def oscillation(kappa: float, nu_l: float, nu_g: float = 0.2, L_: int = 120, rmax: float = 30.0,
                rmin: float = 27.0, steps: int = 12000, every: int = 10, A: float = -0.3,
                sigma: float = None, precision: int = L.LBM_FP32) -> Dict:
    """Period of the n = 2 mode of an elliptic cylinder, against Eq. 30."""
    eos = pr_eos()
    rl, rg = pr_coexistence(0.0, A)
    lat = L.Lattice(L_, L_, precision)
    lat.set_params(eos, A, kappa, G=-1.0, s=S_ONES, rho_ref=rg)
    lat.set_viscosity(nu_g, nu_l, rg, rl)
    lat.init_density(I.ellipse_density(L_, L_, rmax, rmin, rl, rg, width=4.0))
    lat.use_graphs(True)
    lat.autotune(40)
    t, D = [], []
    for n in range(steps // every + 1):
        if n:
            lat.step(every)
        t.append(n * every)
        D.append(deformation(lat.read_fields(which=("rho",))["rho"], rg))
    lat.close()
    t = np.array(t, dtype=np.float64)
    D = np.array(D)
    # zero crossings of the deformation around its final value (linear interpolation)
    base = D[-len(D) // 5:].mean()
    z = D - base
    cross = [t[i] - z[i] * (t[i + 1] - t[i]) / (z[i + 1] - z[i]) for i in range(len(z) - 1)
             if z[i] == 0 or (z[i] < 0) != (z[i + 1] < 0)]
    halves = np.diff(cross)
    period = float(2 * np.mean(halves[:4])) if len(halves) else float("nan")
    R0 = math.sqrt(rmax * rmin)
    theory = 2 * math.pi * math.sqrt(rl * R0 ** 3 / (6.0 * sigma)) if sigma else float("nan")
    return {"kappa": kappa, "nu_l": nu_l, "nu_g": nu_g, "period": period, "theory": theory,
            "rel_err": period / theory - 1 if sigma else float("nan"), "crossings": [float(c) for c in cross[:8]],
            "rho_l": rl, "rho_g": rg, "sigma": sigma}


def main(argv=None):
    ap = argparse.ArgumentParser(description="the paper's experiments on the GPU path")
    ap.add_argument("--method1", action="store_true")
    ap.add_argument("--pr-laplace", action="store_true")
    ap.add_argument("--oscillation", action="store_true")
    args = ap.parse_args(argv)
    out = {}
    if args.method1:
        out["method1"] = method1()
    if args.pr_laplace or args.oscillation:
        pl = pr_laplace(kappas=(-1.0, 0.0, 0.5, 0.9, 0.99))
        out["pr_laplace"] = pl
    if args.oscillation:
        osc = []
        for k in (-1.0, 0.0, 0.5):
            sig = out["pr_laplace"]["fits"].get(k, {}).get("sigma")
            for nl in (0.05, 0.1):
                osc.append(oscillation(k, nl, sigma=sig, steps=14000 if k < 0.5 else 20000))
        out["oscillation"] = osc
    print(json.dumps(out))


if __name__ == "__main__":
    main()
