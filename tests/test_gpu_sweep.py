"""Batched droplet sweeps on the GPU: Laplace-law fits against the oracle,
and the batched launch against one-by-one runs."""
import warnings

import numpy as np
import pytest

import lbm_inputs as I
import oracle as O
from oracle import analysis as An

warnings.filterwarnings("ignore", category=Warning, module="scipy")

pytestmark = pytest.mark.gpu
S_CFG = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]


@pytest.fixture(scope="module")
def SW():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_7228_gb300 import sweep
    return sweep


def oracle_sample(p, f, N, R0, gap=10.0):
    """The sweep's Laplace sampling on the oracle: a first pass with discs
    from R0 gives the equimolar radius R, the second samples r <= R/2 and
    r >= R + gap."""
    rho = O.macro(p, f)[0]
    d = An.pressure_jump(p, rho, N / 2, N / 2, R0 / 2, R0 + gap)
    R = d["R_eq"]
    return An.pressure_jump(p, rho, N / 2, N / 2, R / 2, R + gap) if R > 0 else d


def oracle_laplace(kappa, radii, N, steps, tr=0.7, A=-0.85, gap=10.0, window=(2000, 20)):
    """The oracle's sigma with the sweep's sampling: Delta p and R_eq are the
    means over the last window[0] steps, one sample every window[1]."""
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A, kappa=kappa, s=list(S_CFG))
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, tr * Tc)
    rg, rl, _ = An.maxwell(p)
    span, every = window
    dps, Rs = [], []
    for R in radii:
        f = O.init_equilibrium(I.droplet_density(N, N, R, rl, rg))
        O.step(p, f, steps - span)
        samples = []
        for k in range(span // every + 1):
            if k:
                O.step(p, f, every)
            samples.append(oracle_sample(p, f, N, R, gap))
        dps.append(np.mean([d["dp"] for d in samples]))
        Rs.append(np.mean([d["R_eq"] for d in samples]))
    return An.laplace_fit(dps, Rs)


def test_laplace_sweep_matches_oracle_and_kappa_law(SW):
    """sigma from the batched FP32 sweep within 1e-3 of the FP64 oracle's
    (both sampled as the mean over the last 2000 steps), r^2 >= 0.999, and
    sigma(0.5)/sigma(0) within 8 % of 1 - kappa: Eq. 28 is the leading order
    of a Taylor expansion, and this Carnahan-Starling interface (2-3 nodes
    wide) is sharper than the paper's K = 0.3 van der Waals one, where the
    oracle lands within 3 % (measured here: 5.4 %)."""
    radii = (10, 14, 18)
    fits, info = SW.laplace_sweep(radii=radii, kappas=(0.0, 0.3, 0.5), t_over_tc=(0.7,), L_=64, steps=4000,
                                  autotune=False)
    by_k = {f.kappa: f for f in fits}
    assert set(by_k) == {0.0, 0.3, 0.5}
    assert all(f.r2 >= 0.999 for f in fits)
    sig_o, _, r2_o = oracle_laplace(0.3, radii, 64, 4000)
    assert abs(by_k[0.3].sigma / sig_o - 1) <= 1e-3
    assert abs(by_k[0.5].sigma / by_k[0.0].sigma / 0.5 - 1) <= 0.08


def test_batched_equals_sequential(SW):
    drops = [SW.Droplet(L, 0.25 * L, tr, -0.85, k) for L, tr, k in
             ((64, 0.7, 0.1), (96, 0.75, 0.4), (128, 0.65, 0.0), (48, 0.8, 0.6))]
    seq = [SW.Droplet(d.L, d.radius, d.t_over_tc, d.A, d.kappa) for d in drops]
    SW.run_batch(drops, 300, autotune=True)
    SW.run_sequential(seq, 300)
    for a, b in zip(drops, seq):
        assert a.status == 0 and b.status == 0
        assert a.dp == b.dp and a.R_eq == b.R_eq and a.umax == b.umax


def test_laplace_sweep_fp32_matches_fp64_at_full_size(SW):
    """The Laplace-law sweep at its full size (256^2, R0 = 20..60, 3e4
    steps) for T = 0.7 Tc and kappa in {0, 0.5}: the FP32 sweep's sigma is
    within 1e-3 of the FP64 sweep's, every fit has r^2 >= 0.999, the
    coexistence densities agree within 1e-3, Eq. 28's kappa law holds within
    8 %, and both precisions match the FP64 oracle's run of the same sweep
    (stored by a script that calls only the oracle).  Delta p is the mean over the last 2000 steps: one instant's
    sample carries the gas's acoustic standing waves, which differ in phase
    between the two precisions (up to 3e-3 of the R0 = 60 drop's Delta p)."""
    radii = (20, 30, 40, 50, 60)
    kw = dict(radii=radii, kappas=(0.0, 0.5), t_over_tc=(0.7,), L_=256, steps=30000)
    f32, _ = SW.laplace_sweep(precision=1, **kw)
    f64, _ = SW.laplace_sweep(precision=2, **kw)
    b32 = {f.kappa: f for f in f32}
    b64 = {f.kappa: f for f in f64}
    assert set(b32) == set(b64) == {0.0, 0.5}
    for k in (0.0, 0.5):
        a, b = b32[k], b64[k]
        assert len(a.radii) == len(b.radii) == 5
        assert a.r2 >= 0.999 and b.r2 >= 0.999
        assert abs(a.sigma / b.sigma - 1) <= 1e-3, (k, a.sigma, b.sigma)
        assert abs(a.rho_l / b.rho_l - 1) <= 1e-3 and abs(a.rho_g / b.rho_g - 1) <= 1e-3
    assert abs(b32[0.5].sigma / b32[0.0].sigma / 0.5 - 1) <= 0.08
    # the same sweep on the FP64 oracle (tests/golden/make_laplace_oracle.py,
    # sampled the same way): FP64 within 1e-6, FP32 within 1e-3
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "laplace_oracle_256.json")) as fh:
        ref = json.load(fh)
    assert ref["L"] == 256 and ref["steps"] == 30000 and ref["window"] == [2000, 20]
    for k in (0.0, 0.5):
        o = ref["fits"][str(k)]
        assert o["r2"] >= 0.999
        assert abs(b64[k].sigma / o["sigma"] - 1) <= 1e-6, (k, b64[k].sigma, o["sigma"])
        assert abs(b32[k].sigma / o["sigma"] - 1) <= 1e-3, (k, b32[k].sigma, o["sigma"])
        assert abs(b32[k].rho_l / o["rho_l"] - 1) <= 1e-3 and abs(b32[k].rho_g / o["rho_g"] - 1) <= 1e-3


def test_trace_of_a_sweep(SW, tmp_path):
    """The JSON-lines trace of a sweep: one record per instance every 100
    steps, with the FP64 reductions of the step: mass conserved to 1e-6 over
    400 steps (the FP32 stored populations round every step; measured
    1.8e-7 here), momentum near zero for a resting drop."""
    import json
    path = tmp_path / "trace.jsonl"
    drops = [SW.Droplet(64, 12.0, 0.7, -0.85, k) for k in (0.0, 0.3, 0.5)]
    SW.run_batch(drops, 400, autotune=False, schedule=(0, 3), trace=str(path), trace_every=100)
    recs = [json.loads(l) for l in path.read_text().splitlines()]
    assert [(r["step"], r["instance"]) for r in recs] == [(s, i) for s in (100, 200, 300, 400) for i in range(3)]
    for i in range(3):
        mass = [r["mass"] for r in recs if r["instance"] == i]
        assert all(r["status"] == 0 for r in recs if r["instance"] == i)
        assert max(abs(m / mass[0] - 1) for m in mass) < 1e-6
        assert all(abs(r["mom_x"]) < 1e-6 * mass[0] and r["ke"] > 0 for r in recs if r["instance"] == i)
