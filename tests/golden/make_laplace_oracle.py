"""Writes tests/golden/laplace_oracle_256.json: the FP64 oracle's Laplace-law
sweep at the full size of the Laplace-sweep workload for T = 0.7 Tc and
kappa in {0, 0.5}: 256^2 periodic, droplets of R0 = 20, 30, 40, 50, 60 at
the centre between the Maxwell densities (tanh width 2), Carnahan-Starling
a = 1, b = 4, R = 1, A = -0.85, s = (1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1, 1),
3x10^4 steps.  Delta p, R_eq and the phase densities are the means over the
last 2000 steps, one sample every 20 (the equimolar radius R from a first
pass, then p_in over r <= R/2 and p_out over r >= R + 10); sigma is the
least-squares slope of Delta p against 1/R_eq (Eq. 22).  Calls only oracle/ (its OpenMP build: same bits as the serial
one); about 2x10^10 lattice updates, some minutes on a many-core host.

  python tests/golden/make_laplace_oracle.py [threads]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lbm_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
from oracle import analysis as An  # noqa: E402

L, STEPS, SPAN, EVERY, GAP = 256, 30000, 2000, 20, 10.0
RADII, KAPPAS, TR, A = (20, 30, 40, 50, 60), (0.0, 0.5), 0.7, -0.85
S = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]


def drop(kappa, R, threads):
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A, kappa=kappa, s=list(S))
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, TR * Tc)
    rg, rl, _ = An.maxwell(p)
    f = O.init_equilibrium(I.droplet_density(L, L, float(R), rl, rg))
    O.step(p, f, STEPS - SPAN, threads=threads)
    samples = []
    for k in range(SPAN // EVERY + 1):
        if k:
            O.step(p, f, EVERY, threads=threads)
        rho = O.macro(p, f)[0]
        d = An.pressure_jump(p, rho, L / 2, L / 2, R / 2, R + GAP)   # R_eq, then discs that follow it
        samples.append(An.pressure_jump(p, rho, L / 2, L / 2, d["R_eq"] / 2, d["R_eq"] + GAP))
    mean = {key: float(np.mean([d[key] for d in samples])) for key in ("dp", "R_eq", "rho_in", "rho_out")}
    mean["R_drift"] = (samples[-1]["R_eq"] - samples[0]["R_eq"]) / samples[-1]["R_eq"]
    return mean


def main(threads):
    out = {"what": __doc__.split("\n\n")[0], "command": "python tests/golden/make_laplace_oracle.py",
           "L": L, "steps": STEPS, "window": [SPAN, EVERY], "t_over_tc": TR, "A": A, "s": S, "fits": {}}
    t0 = time.time()
    for kappa in KAPPAS:
        drops = [drop(kappa, R, threads) for R in RADII]
        sigma, icpt, r2 = An.laplace_fit([d["dp"] for d in drops], [d["R_eq"] for d in drops])
        out["fits"][str(kappa)] = {"sigma": sigma, "intercept": icpt, "r2": r2,
                                   "rho_l": float(np.mean([d["rho_in"] for d in drops])),
                                   "rho_g": float(np.mean([d["rho_out"] for d in drops])),
                                   "drops": {str(R): d for R, d in zip(RADII, drops)}}
        print(kappa, sigma, r2, "%.0f s" % (time.time() - t0), flush=True)
    with open(os.path.join(HERE, "laplace_oracle_256.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1))
