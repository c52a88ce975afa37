"""Parameter sweeps over many droplets in one batched launch per step.

Host orchestration over the C ABI only: every lattice update, reduction and
least-squares fit runs in liblbm.so.  Two drivers:

- ``laplace_sweep``: static droplets of several radii for each (T/Tc, kappa);
  sigma is the slope of Delta p against 1/R_eq (Laplace's law, Eq. 22), with
  the coexistence densities and the peak spurious velocity per instance.
- ``batched_sweep``: uneven square domains stepped together, one launch per
  step for up to 64 instances (their tensor maps and tile counts in the
  kernel's argument block, CUDA-graph replay, tile shape and CTA schedule
  picked by ``lbm_autotune``), timed against running the same instances one
  after another.

Run as ``python -m paper_1412_7228_gb300.sweep --help``.
"""
import argparse
import functools
import json
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

import lbm_inputs as I

from . import lbm as L

S_DEFAULT = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
CS = dict(kind=L.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)


@functools.lru_cache(maxsize=None)
def _cs_state(t_over_tc: float) -> Tuple[float, float, float]:
    eos = L.Eos(**CS)
    _, Tc, _ = L.lbm_eos_critical(eos)
    eos.T = t_over_tc * Tc
    rg, rl, _ = L.lbm_eos_maxwell(eos)
    return eos.T, rg, rl


def cs_eos(t_over_tc: float) -> Tuple[L.Eos, float, float]:
    """Carnahan-Starling law at T = t_over_tc * Tc and its Maxwell densities."""
    T, rg, rl = _cs_state(float(t_over_tc))
    return L.Eos(T=T, **CS), rg, rl


@dataclass
class Droplet:
    L: int
    radius: float
    t_over_tc: float
    A: float
    kappa: float
    # results
    dp: float = float("nan")
    R_eq: float = float("nan")
    rho_l: float = float("nan")
    rho_g: float = float("nan")
    umax: float = float("nan")
    status: int = 0
    R_drift: float = float("nan")   # relative change of R_eq over the sampling window
    n_samples: int = 0

    @property
    def sigma_single(self) -> float:
        """Delta p * R_eq of this droplet alone (Eq. 22)."""
        return self.dp * self.R_eq


def _setup(batch: L.Batch, i: int, d: Droplet, s=S_DEFAULT):
    eos, rg, rl = cs_eos(d.t_over_tc)
    L.Batch.set_params(batch, i, eos, d.A, d.kappa, G=-1.0, s=s, rho_ref=rg)
    L.Batch.init_density(batch, i, I.droplet_density(d.L, d.L, d.radius, rl, rg))


R_OUT_GAP = 10.0   # p_out is sampled at r >= R + 10 (the gas beyond the interface)
# Laplace sampling window: the mean of Delta p (and of R_eq and the phase
# densities) over the last WINDOW_STEPS steps, sampled every WINDOW_EVERY
# (each sample as in _sample).
# A static drop keeps acoustic standing waves in the gas between it and its
# periodic images (periods of 60-270 steps at 256^2, decaying over ~10^4
# steps); one instant's Delta p carries them (up to 3 % of Delta p for
# R0 = 60 at 3e4 steps), the window mean leaves the Laplace pressure.
WINDOW_STEPS, WINDOW_EVERY = 2000, 20


def _sample(batch: L.Batch, i: int, d: Droplet) -> Dict:
    """Laplace sampling of droplet i with discs that follow the drop's size:
    a first pass (p_in over r <= R0/2, p_out over r >= R0 + 10) gives its
    equimolar radius R, the second samples p_in over r <= R/2 and p_out over
    r >= R + 10, so the inner disc stays well inside the liquid when a small
    drop has shrunk (at 0.8 Tc an R0 = 20 drop settles at R = 12.6, and a
    disc of radius 10 would reach into its interface)."""
    c = d.L / 2.0
    m = batch.measure(i, c, c, d.radius / 2.0, d.radius + R_OUT_GAP)
    R = m["R_eq"]
    if not (R > 0 and np.isfinite(R)):
        return m
    return batch.measure(i, c, c, R / 2.0, R + R_OUT_GAP)


def _harvest(batch: L.Batch, i: int, d: Droplet, acc: Optional[List[Dict]] = None):
    """Results of droplet i: the window means of acc (its samples) when
    given, else one sample now."""
    d.status = batch.status(i)
    if d.status != L.LBM_OK:
        return
    samples = acc if acc else [_sample(batch, i, d)]
    mean = lambda k: float(np.mean([m[k] for m in samples]))
    d.dp, d.R_eq, d.rho_l, d.rho_g = mean("dp"), mean("R_eq"), mean("rho_in"), mean("rho_out")
    d.R_drift = (samples[-1]["R_eq"] - samples[0]["R_eq"]) / max(abs(samples[-1]["R_eq"]), 1e-300)
    d.n_samples = len(samples)
    d.umax = batch.stats(i)["umax"]


def _wait():
    """Wait for the device (no status check: unstable instances are reported
    per instance by the caller)."""
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()


class Trace:
    """Per-run JSON-lines trace of the FP64 reductions (lbm_batch_stats):
    every `every` steps one line per instance with the step, the instance,
    its mass, momentum, kinetic energy, peak speed and status, so that a long
    sweep leaves a record of conservation and of spurious currents."""

    def __init__(self, path: str, every: int):
        if every < 1:
            raise ValueError("the trace interval must be at least one step")
        self.fh = open(path, "a")
        self.every = every
        self.seconds = 0.0

    def record(self, batch: L.Batch, step: int):
        _wait()   # the steps so far belong to the stepping time, not to the trace
        t = time.perf_counter()
        for i in range(batch.n):
            st = batch.status(i)
            rec = {"step": step, "instance": i, "status": st}
            if st == L.LBM_OK:
                rec.update(batch.stats(i))
            self.fh.write(json.dumps(rec) + "\n")
        self.fh.flush()
        self.seconds += time.perf_counter() - t

    def close(self):
        self.fh.close()


def _advance(batch: L.Batch, n: int, done: int, trace: Optional[Trace]) -> int:
    """Step n times; with a trace, stop at every multiple of its interval to
    record it.  Returns the steps done."""
    if trace is None:
        batch.step(n)
        return done + n
    end = done + n
    while done < end:
        k = min(end, (done // trace.every + 1) * trace.every) - done
        batch.step(k)
        done += k
        if done % trace.every == 0:
            trace.record(batch, done)
    return done


def run_batch(droplets: Sequence[Droplet], steps: int, precision: int = L.LBM_FP32, autotune: bool = True,
              graphs: bool = True, s=S_DEFAULT, schedule: Optional[Tuple[int, int]] = None,
              window: Optional[Tuple[int, int]] = None, trace: Optional[str] = None,
              trace_every: int = 1000) -> Dict:
    """Step every droplet together; fill in the per-droplet results.
    schedule: (tile configuration, CTA schedule) instead of autotuning.
    window: (span, every): Laplace sampling averaged over the last `span`
    steps, one sample every `every` steps (None: one sample at the end).
    trace: append a JSON-lines record of every instance's reductions every
    trace_every steps to this file (Trace)."""
    import torch
    batch = L.Batch([d.L for d in droplets], [d.L for d in droplets], precision)
    for i, d in enumerate(droplets):
        _setup(batch, i, d, s)
    if graphs:
        batch.use_graphs(True)   # first: the autotuner times the schedules as they will run
    tune = None
    if schedule is not None:
        batch.set_schedule(*schedule)
    elif autotune:
        # enough steps that the multi-step schedule's launch is measured over
        # many steps, as a long sweep runs it
        tune = batch.autotune(40)
    acc = None
    span, every = window if window else (0, 1)
    if span >= steps or span % every:
        raise ValueError("the window must be a whole number of sampling intervals shorter than the run")
    tr = Trace(trace, trace_every) if trace else None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sample_s = 0.0
    done = _advance(batch, steps - span, 0, tr)
    if window:
        acc = [[] for _ in droplets]
        for k in range(span // every + 1):
            if k:
                done = _advance(batch, every, done, tr)
            _wait()   # the steps so far belong to the stepping time, not to the sampling
            t1 = time.perf_counter()
            for i, d in enumerate(droplets):
                acc[i].append(_sample(batch, i, d))
            sample_s += time.perf_counter() - t1
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0 - sample_s - (tr.seconds if tr else 0.0)
    if tr:
        tr.close()
    launches = batch.kernel_launches
    for i, d in enumerate(droplets):
        _harvest(batch, i, d, acc[i] if acc else None)
    batch.clear_status()
    batch.close()
    nodes = sum(d.L * d.L for d in droplets)
    return {"seconds": dt, "mlups": nodes * steps / dt / 1e6, "tune": tune, "launches": launches,
            "sampling_seconds": sample_s}


def run_sequential(droplets: Sequence[Droplet], steps: int, precision: int = L.LBM_FP32, graphs: bool = True,
                   s=S_DEFAULT) -> Dict:
    """The same droplets one after another, one context each."""
    import torch
    total = 0.0
    for d in droplets:
        lat = L.Lattice(d.L, d.L, precision)
        _setup(lat, 0, d, s)
        if graphs:
            lat.use_graphs(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(steps)
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
        _harvest(lat, 0, d)
        lat.close()
    nodes = sum(d.L * d.L for d in droplets)
    return {"seconds": total, "mlups": nodes * steps / total / 1e6}


@dataclass
class LaplaceFit:
    t_over_tc: float
    kappa: float
    sigma: float
    intercept: float
    r2: float
    rho_l: float
    rho_g: float
    umax: float
    radii: List[float] = field(default_factory=list)


def in_equilibrium(d: Droplet, max_drift: float = 1e-3) -> bool:
    """Laplace's law holds for drops at equilibrium: a drop is used when it
    is stable, still a liquid drop (its core denser than the gas around it
    by half the Maxwell density gap) and, when sampled over a window, its
    equimolar radius moved by less than max_drift there (an evaporating drop
    keeps shrinking)."""
    if d.status != L.LBM_OK or not (np.isfinite(d.dp) and np.isfinite(d.R_eq) and d.R_eq > 0):
        return False
    _, rg, rl = cs_eos(d.t_over_tc)
    if not d.rho_l - d.rho_g >= 0.5 * (rl - rg):
        return False
    return d.n_samples <= 1 or abs(d.R_drift) <= max_drift


def laplace_sweep(radii=(20, 30, 40, 50, 60), kappas=(0.0, 0.1, 0.3, 0.5), t_over_tc=(0.6, 0.7, 0.8), L_=256,
                  steps=30000, A=-0.85, precision=L.LBM_FP32, autotune=True,
                  window=(WINDOW_STEPS, WINDOW_EVERY), trace: Optional[str] = None,
                  trace_every: int = 1000) -> Tuple[List[LaplaceFit], Dict]:
    drops = [Droplet(L_, float(R), tr, A, k) for tr in t_over_tc for k in kappas for R in radii]
    info = run_batch(drops, steps, precision, autotune=autotune, window=window, trace=trace,
                     trace_every=trace_every)
    info["droplets"] = [{k: getattr(d, k) for k in ("radius", "t_over_tc", "kappa", "dp", "R_eq", "rho_l", "rho_g",
                                                     "umax", "status", "R_drift")} for d in drops]
    fits = []
    for tr in t_over_tc:
        for k in kappas:
            grp = [d for d in drops if d.t_over_tc == tr and d.kappa == k and in_equilibrium(d)]
            if len(grp) < 2:
                continue
            sigma, icpt, r2 = L.lbm_laplace_fit([d.dp for d in grp], [d.R_eq for d in grp])
            fits.append(LaplaceFit(tr, k, sigma, icpt, r2, float(np.mean([d.rho_l for d in grp])),
                                   float(np.mean([d.rho_g for d in grp])), float(max(d.umax for d in grp)),
                                   [d.R_eq for d in grp]))
    return fits, info


def sweep_droplets(n=64, seed=7228, sizes=(128, 256, 512, 1024), A_shift=-0.7) -> List[Droplet]:
    """The batched uneven sweep's instances.  A is drawn from U[-0.2, -0.1]
    shifted by A_shift: with the forcing of Eqs. 5-6, eps = -2A of Eq. 17 so
    small leaves the Carnahan-Starling law without a coexistence state of
    positive pressure below about 0.75 Tc, while A near -0.85 keeps it within
    0.2 % (liquid) of Maxwell's densities at 0.6-0.8 Tc."""
    return [Droplet(s.L, s.radius, s.T_over_Tc, s.A + A_shift, s.kappa)
            for s in I.sweep_instances(n, seed, sizes)]


def main(argv=None):
    ap = argparse.ArgumentParser(description="batched droplet sweeps on the GPU")
    ap.add_argument("--laplace", action="store_true", help="Laplace-law sweep (256^2, 5 radii x 4 kappa x 3 T)")
    ap.add_argument("--batched", action="store_true", help="64 uneven instances, batched vs sequential")
    ap.add_argument("--uniform", type=int, default=None, metavar="L",
                    help="time --n droplets of L^2 (R0 = 0.2 L, 0.7 Tc, A = -0.85, kappa = 0.3) stepped together: "
                         "tile and schedule autotuned, graphs on; or with --tile/--schedule as given and without "
                         "graphs (each launch as a profiler sees it)")
    ap.add_argument("--tile", type=int, default=None)
    ap.add_argument("--schedule", type=int, default=None)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--trace", default=None, metavar="PATH",
                    help="append a JSON-lines trace of every instance's mass, momentum, kinetic energy and peak "
                         "speed (Laplace sweep)")
    ap.add_argument("--trace-every", type=int, default=1000)
    args = ap.parse_args(argv)
    prec = L.LBM_FP32 if args.precision == "fp32" else L.LBM_FP64
    if args.laplace:
        fits, info = laplace_sweep(steps=args.steps or 30000, precision=prec, trace=args.trace,
                                   trace_every=args.trace_every)
        out = {"sweep": "laplace", "precision": args.precision, "seconds": info["seconds"], "mlups": info["mlups"],
               "fits": [f.__dict__ for f in fits], "droplets": info.get("droplets")}
        print(json.dumps(out))
    if args.uniform:
        steps = args.steps or 2000
        drops = [Droplet(args.uniform, 0.2 * args.uniform, 0.7, -0.85, 0.3) for _ in range(args.n)]
        forced = args.tile is not None or args.schedule is not None
        sched = (args.tile or 0, args.schedule or 0) if forced else None
        r = run_batch(drops, steps, prec, graphs=not forced, schedule=sched)
        tile, schedule = sched if forced else tuple(r["tune"][:2])
        print(json.dumps({"sweep": "uniform", "instances": args.n, "L": args.uniform, "steps": steps,
                          "precision": args.precision, "tile": tile, "schedule": schedule,
                          "seconds": r["seconds"], "mlups": r["mlups"], "launches": r["launches"],
                          "unstable": sum(d.status != 0 for d in drops)}))
    if args.batched:
        steps = args.steps or 20000
        drops = sweep_droplets(args.n)
        b = run_batch(drops, steps, prec)
        seq_drops = sweep_droplets(args.n)
        q = run_sequential(seq_drops, steps, prec)
        agree = max(abs(a.dp - c.dp) / max(abs(c.dp), 1e-30) for a, c in zip(drops, seq_drops)
                    if a.status == 0 and c.status == 0)
        out = {"sweep": "batched", "instances": len(drops), "steps": steps, "precision": args.precision,
               "batched_s": b["seconds"], "sequential_s": q["seconds"], "speedup": q["seconds"] / b["seconds"],
               "batched_mlups": b["mlups"], "sequential_mlups": q["mlups"], "tune": b["tune"],
               "unstable": sum(d.status != 0 for d in drops), "max_rel_dp_diff": agree}
        print(json.dumps(out))


if __name__ == "__main__":
    main()
