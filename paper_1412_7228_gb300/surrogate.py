"""Learned surrogate over the simulation: data, training, inverse, check.

1. Data: static droplets with (T/Tc, A, kappa) drawn by the batched sweep's
   generator, all on one geometry (L x L periodic, R0 = 0.2 L), simulated
   together in one batched launch per step.  Targets per droplet: sigma =
   Delta p * R_eq (Laplace's law, Eq. 22), rho_l, rho_g and the peak spurious
   velocity.  Droplets that went unstable are dropped.
2. Training: the library's CUDA kernels (lbm_mlp_train), MSE on
   standardised targets; sigma and the spurious velocity span an order of
   magnitude, so the network learns their logarithms (relative accuracy),
   with a learning rate that steps down over three phases.
3. Inverse: for requested sigma values at a fixed (T/Tc, A), the GPU
   bisection (lbm_mlp_invert_kappa) picks kappa.
4. Check: every pick is re-simulated on the same geometry; its measured
   sigma is reported against the request.  The same requests are also
   answered without the network, by Eq. 28's sigma(kappa) = (1 - kappa)
   sigma(0) from one extra simulation at kappa = 0, for comparison.

Host orchestration over the C ABI; ``python -m paper_1412_7228_gb300.surrogate``.
"""
import argparse
import json
import time
from typing import Dict, List, Tuple

import numpy as np

import lbm_inputs as I

from . import lbm as L
from .sweep import Droplet, run_batch


def sample_params(n: int, seed: int = 1, A_shift: float = -0.7) -> np.ndarray:
    """(T/Tc, A, kappa) of n droplets from the batched sweep's generator."""
    inst = I.sweep_instances(n, seed)
    return np.array([[s.T_over_Tc, s.A + A_shift, s.kappa] for s in inst])


def simulate(params: np.ndarray, L_: int, steps: int, chunk: int = 1024, precision: int = L.LBM_FP32
             ) -> Tuple[np.ndarray, np.ndarray, Dict]:
    """Targets (sigma, rho_l, rho_g, umax) of droplets with the given
    (T/Tc, A, kappa), chunk droplets per batched launch.  Returns (targets,
    ok-mask, timing)."""
    Y = np.full((len(params), 4), np.nan)
    ok = np.zeros(len(params), dtype=bool)
    seconds, lups = 0.0, 0.0
    for c0 in range(0, len(params), chunk):
        drops = [Droplet(L_, 0.2 * L_, float(t), float(a), float(k)) for t, a, k in params[c0:c0 + chunk]]
        info = run_batch(drops, steps, precision)   # tile and schedule autotuned: a few seconds per chunk
        seconds += info["seconds"]
        lups += len(drops) * L_ * L_ * steps
        for i, d in enumerate(drops):
            if d.status == 0 and np.isfinite(d.dp) and d.dp > 0:
                ok[c0 + i] = True
                Y[c0 + i] = [d.sigma_single, d.rho_l, d.rho_g, d.umax]
    return Y, ok, {"seconds": seconds, "mlups": lups / seconds / 1e6 if seconds > 0 else 0.0}


def to_net(Y: np.ndarray) -> np.ndarray:
    """Targets as the network learns them: (log sigma, rho_l, rho_g, log umax)."""
    Z = np.array(Y, dtype=np.float64)
    Z[:, 0] = np.log(Z[:, 0])
    Z[:, 3] = np.log(Z[:, 3])
    return Z


def from_net(Z: np.ndarray) -> np.ndarray:
    Y = np.array(Z, dtype=np.float64)
    Y[:, 0] = np.exp(Y[:, 0])
    Y[:, 3] = np.exp(Y[:, 3])
    return Y


def train(X: np.ndarray, Y: np.ndarray, epochs: int = 600, batch: int = 128, lr: float = 3e-3, seed: int = 0
          ) -> Tuple[L.Mlp, np.ndarray]:
    Z = to_net(Y)
    mlp = L.Mlp(max_samples=max(len(X), 64), seed=seed)
    mlp.fit_normalization(X, Z)
    losses = []
    for frac, f in ((0.5, 1.0), (0.3, 0.3), (0.2, 0.1)):
        losses.append(mlp.train(X, Z, epochs=max(1, int(epochs * frac)), batch=batch, lr=lr * f, seed=seed + 1))
    return mlp, np.concatenate(losses)


def predict(mlp: L.Mlp, X: np.ndarray) -> np.ndarray:
    return from_net(mlp.predict(X))


def requests(mlp: L.Mlp, Y_ok: np.ndarray, X_ok: np.ndarray, n: int = 16, k_lo: float = 0.0, k_hi: float = 0.6
             ) -> Tuple[float, float, np.ndarray]:
    """n sigma targets spread evenly over the part of the data's 5-95 %
    sigma range that kappa in [k_lo, k_hi] can reach at the data's median
    (T/Tc, A) (1 % inside its ends)."""
    tr, A = float(np.median(X_ok[:, 0])), float(np.median(X_ok[:, 1]))
    lo, hi = np.percentile(Y_ok[:, 0], [5, 95])
    s_hi, s_lo = predict(mlp, np.array([[tr, A, k_lo], [tr, A, k_hi]]))[:, 0]
    lo, hi = max(lo, s_lo * 1.01), min(hi, s_hi * 0.99)
    return tr, A, np.linspace(lo, hi, n)


def pipeline(n: int = 2000, L_: int = 256, steps: int = 40000, epochs: int = 600, n_req: int = 16,
             seed: int = 1, save: str = None) -> Dict:
    X = sample_params(n, seed)
    t0 = time.perf_counter()
    Y, ok, sim = simulate(X, L_, steps)
    t_data = time.perf_counter() - t0
    if save:
        np.savez(save, X=X, Y=Y, ok=ok)
    Xo, Yo = X[ok], Y[ok]
    mlp, losses = train(Xo, Yo, epochs=epochs)
    tr, A, targets = requests(mlp, Yo, Xo, n_req)
    t1 = time.perf_counter()
    # output 0 is log sigma, which decreases in kappa as sigma does
    kappa = mlp.invert_kappa(np.full(len(targets), tr), np.full(len(targets), A), np.log(targets), 0.0, 0.6)
    t_pick = time.perf_counter() - t1
    picks = np.stack([np.full(len(targets), tr), np.full(len(targets), A), kappa], 1)
    Yv, okv, _ = simulate(picks, L_, steps)
    err = Yv[:, 0] / targets - 1
    # without the network: Eq. 28, sigma(kappa) = (1 - kappa) sigma(0), one simulation at kappa = 0
    Y0, _, _ = simulate(np.array([[tr, A, 0.0]]), L_, steps)
    k_lin = np.clip(1.0 - targets / Y0[0, 0], 0.0, 0.6)
    Yl, okl, _ = simulate(np.stack([np.full(len(targets), tr), np.full(len(targets), A), k_lin], 1), L_, steps)
    err_lin = Yl[:, 0] / targets - 1
    pred = predict(mlp, Xo)
    rel = np.abs(pred / Yo - 1)
    mlp.close()
    return {
        "samples": int(n), "stable": int(ok.sum()), "geometry": "%dx%d periodic, R0 = %.1f, %d steps" % (
            L_, L_, 0.2 * L_, steps),
        "data_seconds": t_data, "data_mlups": sim["mlups"],
        "train_loss_first_last": [float(losses[0]), float(losses[-1])],
        "fit_median_rel_err": {k: float(np.median(rel[:, i])) for i, k in enumerate(("sigma", "rho_l", "rho_g",
                                                                                   "umax"))},
        "request_t_over_tc": tr, "request_A": A, "targets": targets.tolist(), "kappa": kappa.tolist(),
        "pick_seconds": t_pick, "resim_sigma": Yv[:, 0].tolist(), "resim_rel_err": err.tolist(),
        "max_abs_rel_err": float(np.nanmax(np.abs(err))),
        "linear_rule_kappa": k_lin.tolist(), "linear_rule_rel_err": err_lin.tolist(),
        "linear_rule_max_abs_rel_err": float(np.nanmax(np.abs(err_lin))),
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the sigma surrogate and check its kappa picks")
    ap.add_argument("--n", type=int, default=2000)
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--steps", type=int, default=40000,
                    help="steps per droplet; a 256^2 drop with R0 = 51 settles by 30-40k steps")
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--save", default=None, help="write the data set (X, Y, ok) to this .npz")
    args = ap.parse_args(argv)
    print(json.dumps(pipeline(args.n, args.L, args.steps, args.epochs, args.requests, save=args.save)))


if __name__ == "__main__":
    main()
