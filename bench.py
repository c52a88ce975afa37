#!/usr/bin/env python3
"""Throughput of the fused sm_103a pseudo-potential MRT step (MLUPS and
fraction of the HBM roofline), FP32 deviation storage with FP64 beside it.

Workload: spinodal decomposition on one 4096 x 4096 periodic lattice,
rho0 = 0.25 (1 + 0.01 u), u from splitmix64 (seed 14127228),
Carnahan-Starling (a=1, b=4, R=1) at T = 0.7 Tc, A = -0.85, kappa = 0.3,
s = (1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1, 1).  One step = one fused kernel
launch over the whole lattice (density, psi, force, Q, collision, stream).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference implementation
of this method here) on all host cores (its OpenMP build), one step = one
oracle time step on a 512 x 512 periodic sample of the same workload.  Under torchrun (N > 1) each
rank runs its own replica lattice (the method needs no exchange between
independent lattices); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline, FP32 vs FP64 on one GB300, sigma err <= 1e-3"
SEED = 14127228
S_CFG = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0]
A_CFG, KAPPA_CFG, TR_CFG, RHO0 = -0.85, 0.3, 0.7, 0.25
# default tile configurations (indices into lbm_tile_config): the fastest at
# 4096^2 when timed with lbm_autotune, 128 x 16 (FP32) and 64 x 16 (FP64)
TILE_FP32, TILE_FP64 = 0, 5
PEAK_FALLBACK_GBS = 6800.0


def workload_config(nx, ny, precision, extra=None):
    cfg = {
        "workload": "spinodal decomposition %dx%d periodic, Carnahan-Starling a=1 b=4 R=1, T=0.7Tc, "
                    "A=-0.85, kappa=0.3, rho0=0.25(1+0.01u)" % (nx, ny),
        "nx": nx, "ny": ny, "precision": precision,
        "l2": "inputs larger than L2: two %.0f MB population arrays per step" % (
            9 * nx * ny * (4 if precision == "fp32" else 8) / 1e6),
    }
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of every rank's value (the timed region ends when the
    slowest replica ends); the identity on one rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, nodes_per_rank, steps, seconds):
    """Lattice updates of all replicas per second, in millions (weak scaling:
    each rank owns one full lattice)."""
    return world * nodes_per_rank * steps / seconds / 1e6


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


KERNEL_SOURCES = ("lbm_step_kernels.cuh", "lbm_step_f32.cu", "lbm_step_f64.cu", "lbm_step.cu", "lbm_internal.cuh")


def kernel_sources_sha():
    """First 16 hex digits of the SHA-256 of the step kernels' sources (the
    kernel header, the two translation units that instantiate it, the
    dispatch file and the header they all compile, in that order), the key
    under which a committed ncu figure is valid."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1412_7228_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_traffic(prec_name, kernel):
    """Measured DRAM bytes per lattice update of the step kernel from the
    committed ncu summary, valid only for the kernel it names and while the
    kernel sources are unchanged (traffic per node does not depend on the
    domain size once the arrays exceed L2)."""
    sha = kernel_sources_sha()
    path = os.path.join(ROOT, "profiles", "step_%s_4096_traffic.txt" % prec_name)
    try:
        kv = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
    except OSError:
        return None
    if kv.get("kernel_sources_sha256_16") != sha or kv.get("kernel") != kernel:
        return None
    try:
        return float(kv["bytes_per_update"])
    except (KeyError, ValueError):
        return None


def oracle_flops_per_update(law="carnahan_starling"):
    """Floating-point operations of one time step per lattice node of the
    FP64 oracle (its traced build, common subexpressions counted once: the
    method's arithmetic, without the kernel's own refinement steps), as
    committed by tests/golden/make_op_count.py."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_op_count.json")) as fh:
            return float(json.load(fh)["counts"][law]["flops_per_update"])
    except (OSError, KeyError, ValueError):
        return None


def fp64_pipe_profile(kernel):
    """ncu figures of the FP64 step kernel (FP64 pipe utilisation and
    executed FP64 instructions per update), valid only for the kernel the
    committed summary names and while the kernel sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "step_fp64_1024_alu.txt")
    try:
        kv = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
    except OSError:
        return None
    if kv.get("kernel_sources_sha256_16") != kernel_sources_sha() or kv.get("kernel") != kernel:
        return None
    out = {}
    for k in ("fp64_pipe_active", "fp64_inst_per_update"):
        try:
            out[k] = float(kv[k])
        except (KeyError, ValueError):
            pass
    return out or None


def fp64_roofline(mlups, flops_per_s_peak):
    """FP64 step against the measured FP64 peak: the oracle's operations per
    update times the update rate, over the FMA-chain rate of this GPU
    measured in the same run (lbm_fp64_fma_rate)."""
    ops = oracle_flops_per_update()
    if ops is None or not flops_per_s_peak:
        return None
    achieved = ops * mlups * 1e6 / 1e9
    peak = flops_per_s_peak / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
            "peak_kind": "measured", "flops_per_update": ops,
            "flops_from": "oracle operation count per update (tests/golden/oracle_op_count.json)",
            "peak_from": "FP64 FMA chains on every SM, this run (lbm_fp64_fma_rate)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        rows = []
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        load = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in load),
                "reasons": sorted(reasons), "samples": len(load)}


def make_lattice(P, nx, ny, prec, rho0, stream=None):
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = TR_CFG * Tc
    lat = P.Lattice(nx, ny, prec, stream=stream)
    lat.set_params(eos, A_CFG, KAPPA_CFG, G=-1.0, s=S_CFG, rho_ref=RHO0)
    lat.init_density(rho0)
    return lat


GRAPH_STEPS = 2    # lbm_step replays captured graphs of 32, 16, 8, 4 and 2 steps; an odd last step is a plain launch


def graph_use(steps):
    """How lbm_step(steps) issues its work once graphs are on: the steps that
    ran from captured graph replays and those that ran as plain launches."""
    g = steps // GRAPH_STEPS * GRAPH_STEPS
    return {"graphs": g > 0, "graph_steps": g, "plain_launch_steps": steps - g}


def time_steps(torch, lat, steps):
    st = lat.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    lat.step(steps)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1000.0


def plain_method_64(torch, P, steps=10000):
    """The plain-method workload in full on the GPU: a 64x64 static droplet
    (R0 = 15, tanh width 2 between the Maxwell densities), Carnahan-Starling
    at 0.7 Tc, A = -0.85, kappa = 0, 10^4 steps, FP32 and FP64, each with its
    autotuned tile and graphs, timed with CUDA events.  It fits in L2 and
    is latency-bound: wall time, no roofline claim."""
    import lbm_inputs as I
    eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
    _, Tc, _ = P.lbm_eos_critical(eos)
    eos.T = TR_CFG * Tc
    rg, rl, _ = P.lbm_eos_maxwell(eos)
    rho0 = I.droplet_density(64, 64, 15.0, rl, rg)
    out = {"workload": "64x64 static droplet R0 = 15, kappa = 0, 10^4 steps (fits in L2: no roofline claim)"}
    for name, prec in (("fp32", P.LBM_FP32), ("fp64", P.LBM_FP64)):
        lat = P.Lattice(64, 64, prec)
        lat.set_params(eos, A_CFG, 0.0, G=-1.0, s=S_CFG, rho_ref=rg)
        lat.init_density(rho0)
        lat.use_graphs(True)
        k, sch, _ = lat.autotune(40)
        lat.init_density(rho0)
        lat.capture_graphs()
        t = time_steps(torch, lat, steps)
        lat.sync()
        lat.close()
        out[name] = {"seconds": t, "us_per_step": t / steps * 1e6, "mlups": 64 * 64 * steps / t / 1e6,
                     "tile": list(P.lbm_tile_configs(prec)[k]) if sch != 4 else "cluster strips", "schedule": sch}
    return out


def laplace_sweep_fp32():
    """The Laplace-law sweep at its full size in FP32: 60 droplets of 256^2
    (R0 = 20..60, kappa 0 / 0.1 / 0.3 / 0.5, T = 0.6 / 0.7 / 0.8 Tc), 3x10^4
    steps, autotuned batched launches, Laplace sampling averaged over the
    last 2000 steps; sigma from Delta p against 1/R_eq per (T, kappa)."""
    from paper_1412_7228_gb300 import sweep as SW
    fits, info = SW.laplace_sweep()
    return {"workload": "60 droplets of 256^2, 3x10^4 steps, FP32", "stepping_seconds": info["seconds"],
            "mlups": info["mlups"], "tile": list(info["tune"][:2]) if info.get("tune") else None,
            "fits": [{"t_over_tc": f.t_over_tc, "kappa": f.kappa, "sigma": f.sigma, "r2": f.r2, "drops": len(f.radii)}
                     for f in fits]}


def batched_vs_sequential(torch, P, steps, n=64, seed=7228):
    """The batched uneven sweep workload (64 static droplets, L uniform over
    {128, 256, 512, 1024}, R0 = 0.2 L, T/Tc ~ U[0.6, 0.85], kappa ~ U[0, 0.6],
    A ~ U[-0.9, -0.8], FP32) stepped `steps` times, once as one batched
    context (tile shape and schedule autotuned) and once as
    64 one-lattice contexts stepped one after another on one stream (each
    with its own autotuned tile), both from CUDA graphs and both timed with
    CUDA events on their stream.  The results of the two must be the same
    bits (compared through each drop's Laplace sampling)."""
    from paper_1412_7228_gb300 import sweep as SW
    drops = SW.sweep_droplets(n, seed)
    nodes = sum(d.L * d.L for d in drops)
    st = torch.cuda.Stream()
    b = P.Batch([d.L for d in drops], [d.L for d in drops], P.LBM_FP32, stream=st)
    for i, d in enumerate(drops):
        SW._setup(b, i, d)
    b.use_graphs(True)
    tile, sched, _ = b.autotune(40)
    b.step(64)
    b.capture_graphs()
    b.sync()
    t_b = time_steps(torch, b, steps)
    b.sync()
    launches_per_step = (b.kernel_launches) / max(b.steps_done, 1)
    res_b = [b.measure(i, d.L / 2, d.L / 2, d.radius / 2, d.radius + SW.R_OUT_GAP)["dp"] for i, d in enumerate(drops)]
    b.close()

    lats = []
    for d in drops:
        lat = P.Lattice(d.L, d.L, P.LBM_FP32, stream=st)
        SW._setup(lat, 0, d)
        lat.use_graphs(True)
        lat.autotune(40)
        lat.step(64)
        lat.capture_graphs()
        lats.append(lat)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for lat in lats:
        lat.step(steps)
    e1.record(st)
    e1.synchronize()
    t_s = e0.elapsed_time(e1) / 1000.0
    res_s = []
    for lat, d in zip(lats, drops):
        lat.sync()
        res_s.append(lat.measure(0, d.L / 2, d.L / 2, d.radius / 2, d.radius + SW.R_OUT_GAP)["dp"])
        lat.close()
    same = all(x == y for x, y in zip(res_b, res_s))
    cut = "" if steps >= 20000 else " (the configured 20000 steps cut to keep the benchmark short)"
    return {"workload": "%d static droplets, L in {128, 256, 512, 1024}, R0 = 0.2 L, seed %d, FP32, %d steps%s"
                        % (n, seed, steps, cut),
            "nodes": nodes, "steps": steps, "batched_s": t_b, "sequential_s": t_s, "speedup": t_s / t_b,
            "batched_mlups": nodes * steps / t_b / 1e6, "sequential_mlups": nodes * steps / t_s / 1e6,
            "batched_tile": [tile, sched], "batched_launches_per_step": launches_per_step,
            "results_bit_identical": same, "timing": "CUDA events on the shared stream, graphs on both arms"}


def cpu_model(cpuinfo="/proc/cpuinfo"):
    """The host CPU's model name (Linux), for the CPU-baseline record."""
    try:
        with open(cpuinfo) as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key == "model name":
                    return line.split(":", 1)[1].strip()
                if key == "cpu part":   # Arm: the part number (0xd4f = Neoverse V2, as in Grace)
                    part = line.split(":", 1)[1].strip()
                    names = {"0xd4f": "Neoverse V2", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1"}
                    return "Arm %s (part %s)" % (names.get(part, "core"), part)
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_mlups(nx, ny, steps):
    """The FP64 oracle as it stands, single-threaded, on a periodic nx x ny
    sample of the workload."""
    import warnings
    warnings.filterwarnings("ignore")
    import lbm_inputs as I
    import oracle as O
    from oracle import analysis as An
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A_CFG, kappa=KAPPA_CFG, G=-1.0, s=list(S_CFG))
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, TR_CFG * Tc)
    f = O.init_equilibrium(I.spinodal_density(nx, ny, RHO0, 0.01, SEED))
    O.step(p, f, 1)
    t0 = time.perf_counter()
    O.step(p, f, steps)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e6, dt


def cpu_oracle_droplet64(steps=10000):
    """The plain-method workload in full on the FP64 oracle, single thread:
    a 64x64 static droplet (R0 = 15 at the centre, tanh width 2 between the
    Maxwell densities), Carnahan-Starling at 0.7 Tc, A = -0.85, kappa = 0,
    10^4 steps.  Returns (MLUPS, seconds)."""
    import warnings
    warnings.filterwarnings("ignore")
    import lbm_inputs as I
    import oracle as O
    from oracle import analysis as An
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A_CFG, kappa=0.0, G=-1.0, s=list(S_CFG))
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, TR_CFG * Tc)
    rg, rl, _ = An.maxwell(p)
    f = O.init_equilibrium(I.droplet_density(64, 64, 15.0, rl, rg))
    t0 = time.perf_counter()
    O.step(p, f, steps)
    dt = time.perf_counter() - t0
    return 64 * 64 * steps / dt / 1e6, dt


def cpu_oracle_all_cores(nx, ny, steps, threads):
    """The OpenMP build of the FP64 oracle (same bits as the serial one) on
    all host cores, on the same sample as cpu_oracle_mlups."""
    import warnings
    warnings.filterwarnings("ignore")
    import lbm_inputs as I
    import oracle as O
    from oracle import analysis as An
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A_CFG, kappa=KAPPA_CFG, G=-1.0, s=list(S_CFG))
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, TR_CFG * Tc)
    f = O.init_equilibrium(I.spinodal_density(nx, ny, RHO0, 0.01, SEED))
    O.step(p, f, 1, threads=threads)
    t0 = time.perf_counter()
    O.step(p, f, steps, threads=threads)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e6, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import warnings
    warnings.filterwarnings("ignore")
    import lbm_inputs as I
    import oracle as O
    from oracle import analysis as An
    n = 512
    threads = os.cpu_count() or 1
    base = O.Params(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0, A=A_CFG, kappa=KAPPA_CFG, G=-1.0, s=list(S_CFG))
    _, Tc, _ = An.critical_point(base)
    p = An.with_T(base, TR_CFG * Tc)
    f = O.init_equilibrium(I.spinodal_density(n, n, RHO0, 0.01, SEED))
    O.step(p, f, args.warmup, threads=threads)
    t0 = time.perf_counter()
    O.step(p, f, args.steps, threads=threads)
    dt = time.perf_counter() - t0
    mlups = n * n * args.steps / dt / 1e6
    sample = ("%dx%d periodic sample of the workload per step, FP64 oracle on all %d host cores (its OpenMP "
              "build, same bits as the serial one)" % (n, n, threads))
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        # the workload of the arm it is compared with; the oracle computes it in FP64 on a sample
        "config": workload_config(args.nx, args.ny, args.precision, {"sample": "%dx%d" % (n, n), "threads": threads}),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle", "sample": sample,
                         "host_cores": os.cpu_count(), "cpu_model": cpu_model()},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import lbm_inputs as I
    import paper_1412_7228_gb300 as P

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    nx, ny = args.nx, args.ny
    N = nx * ny
    rho0 = I.spinodal_density(nx, ny, RHO0, 0.01, SEED)

    prec = P.LBM_FP32 if args.precision == "fp32" else P.LBM_FP64
    lat = make_lattice(P, nx, ny, prec, rho0)
    if args.autotune:
        k, s, ms = lat.autotune(10)
    else:
        k = args.tile if args.tile is not None else (TILE_FP32 if prec == P.LBM_FP32 else TILE_FP64)
        lat.set_schedule(k, 0)
    tile = P.lbm_tile_configs(prec)[k]
    lat.use_graphs(True)
    launches0 = lat.kernel_launches
    lat.step(args.warmup)
    lat.capture_graphs()   # every graph the timed steps replay, captured outside the timed region
    lat.sync()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        barrier()
        launches_t0 = lat.kernel_launches
        t = time_steps(torch, lat, args.steps)
        barrier()
    launches = lat.kernel_launches - launches_t0
    status_ok = True
    try:
        lat.sync()
    except P.LbmError:
        status_ok = False
    t = max_over_ranks(t, dist, "cuda")
    mlups = whole_job_mlups(ws, N, args.steps, t)
    avg_launch = t / args.steps
    peak, peak_kind = measured_peak()
    bpu = 72 if prec == P.LBM_FP32 else 144
    achieved = bpu * N / avg_launch / 1e9
    kname = (("lbm::k_step_f32<%d,%d,%d,%d,1>" % tuple(tile)) if prec == P.LBM_FP32
             else ("lbm::k_step<double,%d,%d,%d,%d,1>" % tuple(tile)))
    tpu = kernel_traffic(args.precision, kname)
    traffic = tpu * N if tpu is not None else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "bytes_per_update": bpu, "kernel": kname}
    if traffic is not None:
        roof["traffic_bytes_per_update"] = tpu
        roof["traffic_gbs"] = traffic / avg_launch / 1e9
    lat.close()

    # ---- FP64 on the same workload (fewer steps: it is FP64-ALU bound) ----
    fp64 = None
    if not args.no_fp64 and prec == P.LBM_FP32:
        lat64 = make_lattice(P, nx, ny, P.LBM_FP64, rho0)
        lat64.set_schedule(TILE_FP64, 0)
        lat64.use_graphs(True)
        lat64.step(min(args.warmup, 10))
        lat64.capture_graphs()
        lat64.sync()
        k64 = max(32, args.steps // 32)
        with ClockSampler(local) as clk64:
            t64 = time_steps(torch, lat64, k64)
            lat64.sync()
            fma_flops, fma_s = P.lbm.lbm_fp64_fma_rate(4096, lat64.stream.cuda_stream)
        m64 = N * k64 / t64 / 1e6
        fp64 = {"value": m64, "unit": "MLUPS", "steps": k64, "ms_per_step": t64 / k64 * 1000.0,
                "hbm_frac": 144 * N / (t64 / k64) / 1e9 / peak, "bytes_per_update": 144,
                "kernel": "lbm::k_step<double,%d,%d,%d,%d,1>" % tuple(P.lbm_tile_configs(P.LBM_FP64)[TILE_FP64]),
                "fp64_peak_gflops": fma_flops / 1e9, "fp64_peak_launch_ms": fma_s * 1e3, "clocks": clk64.summary()}
        roof64 = fp64_roofline(m64, fma_flops)
        if roof64:
            fp64["roofline"] = roof64
        prof64 = fp64_pipe_profile(fp64["kernel"])
        if prof64:
            fp64["ncu"] = prof64
        lat64.close()

    # ---- the same step on the paper's other synthetic workloads -----------
    # a static droplet (R = 0.2 L between the Maxwell densities) and a flat
    # interface (liquid in the centre half), FP32 and FP64, same lattice size
    others = None
    if not args.no_workloads:
        others = {}
        eos_o = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
        _, Tc_o, _ = P.lbm_eos_critical(eos_o)
        eos_o.T = TR_CFG * Tc_o
        rg, rl, _ = P.lbm_eos_maxwell(eos_o)
        fields = {"droplet": I.droplet_density(nx, ny, 0.2 * min(nx, ny), rl, rg),
                  "flat_interface": I.slab_density(nx, ny, rl, rg, width=4.0)}
        for name, rho_init in fields.items():
            res = {}
            for pname, pr, kk, nsteps in (("fp32", P.LBM_FP32, TILE_FP32, 192), ("fp64", P.LBM_FP64, TILE_FP64, 32)):
                lo = P.Lattice(nx, ny, pr)
                lo.set_schedule(kk, 0)
                lo.set_params(eos_o, A_CFG, KAPPA_CFG, G=-1.0, s=S_CFG, rho_ref=rg)
                lo.init_density(rho_init)
                lo.use_graphs(True)
                lo.step(32)
                lo.capture_graphs()
                lo.sync()
                tt = time_steps(torch, lo, nsteps)
                lo.sync()
                lo.close()
                m = N * nsteps / tt / 1e6
                bb = 72 if pr == P.LBM_FP32 else 144
                res[pname] = {"mlups": m, "hbm_frac": bb * N / (tt / nsteps) / 1e9 / peak, "steps": nsteps}
            others[name] = res
        del fields

    # ---- end to end through the public API with host buffers -------------
    e2e = None
    if not args.no_e2e:
        # fields in the lattice's precision: FP32 lattices take and return float32
        # (lbm_init_density_f32 / lbm_read_fields_f32), FP64 ones float64
        fdt = np.float32 if prec == P.LBM_FP32 else np.float64
        host_rho = torch.from_numpy(rho0.astype(fdt)).pin_memory().numpy()
        out_rho = torch.empty((ny, nx), dtype=torch.float32 if fdt == np.float32 else torch.float64).pin_memory().numpy()
        eos = P.Eos(kind=P.LBM_EOS_CS, a=1.0, b=4.0, R=1.0, K=1.0)
        _, Tc, _ = P.lbm_eos_critical(eos)
        eos.T = TR_CFG * Tc
        lat = P.Lattice(nx, ny, prec)
        lat.set_schedule(k, 0)
        lat.set_params(eos, A_CFG, KAPPA_CFG, G=-1.0, s=S_CFG, rho_ref=RHO0)
        lat.use_graphs(True)
        lat.init_density(host_rho)
        lat.step(args.warmup)
        lat.capture_graphs()
        lat.sync()
        barrier()
        t0 = time.perf_counter()
        lat.init_density(host_rho)
        lat.step(args.steps)
        lat.read_fields(which=("rho",), out={"rho": out_rho}, dtype=fdt)
        t_e2e = time.perf_counter() - t0
        lat.close()
        # the whole job: every replica's updates over the slowest replica's time,
        # and every replica's copies
        t_e2e = max_over_ranks(t_e2e, dist, "cuda")
        esz = np.dtype(fdt).itemsize
        e2e = {"value": whole_job_mlups(ws, N, args.steps, t_e2e), "unit": "MLUPS",
               "h2d_bytes_per_step": ws * esz * N / args.steps, "d2h_bytes_per_step": ws * esz * N / args.steps,
               "what": "lbm_init_density%s from pinned host rho, lbm_step(K), lbm_read_fields%s(rho) to pinned host memory"
                       % (("_f32", "_f32") if esz == 4 else ("", "")) + (", on each of %d ranks" % ws if ws > 1 else "")}

    # ---- the plain-method workload in full: 64^2 droplet, 10^4 steps --------
    plain = None
    if not args.no_workloads:
        plain = plain_method_64(torch, P)

    # ---- the Laplace-law sweep, FP32, at its full size ----------------------
    laplace = None
    if not args.no_sweep:
        laplace = laplace_sweep_fp32()

    # ---- batched uneven sweep against the same lattices one after another ---
    batched = None
    if not args.no_sweep:
        batched = batched_vs_sequential(torch, P, args.sweep_steps)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:   # the CPU baseline: one process, N = 1 only
        cn = args.cpu_n
        m, dt = cpu_oracle_mlups(cn, cn, args.cpu_steps)
        cpu = {"value": m, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": "%d steps of a %dx%d periodic sample of the workload (%.1f s), FP64 single-thread"
                         % (args.cpu_steps, cn, cn, dt),
               "host_cores": os.cpu_count(), "cpu_model": cpu_model()}
        nth = os.cpu_count() or 1
        ma, dta = cpu_oracle_all_cores(cn, cn, args.cpu_steps, nth)
        cpu["all_cores"] = {"value": ma, "unit": "MLUPS", "cores": nth, "seconds": dta,
                            "sample": "the same sample, OpenMP build of the oracle (same bits)"}
        md, dtd = cpu_oracle_droplet64()
        cpu["plain_method_64x64"] = {"value": md, "unit": "MLUPS", "cores": 1, "seconds": dtd,
                                     "sample": "64x64 static droplet R0 = 15, kappa = 0, 10^4 steps: the whole "
                                               "plain-method workload, FP64 oracle, single thread"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1000.0 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == P.LBM_FP32 else "f64",
            "data": "synthetic",
            "config": workload_config(nx, ny, args.precision, dict(
                {"tile": list(tile), "parallelism": "replicas" if ws > 1 else "single"}, **graph_use(args.steps))),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches, "fp64": fp64, "other_workloads": others, "plain_method_64x64": plain,
            "laplace_sweep": laplace, "batched_sweep": batched,
            "status_ok": status_ok,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--tile", type=int, default=None,
                    help="tile configuration index (lbm_tile_config); default %d (FP32) or %d (FP64)"
                         % (TILE_FP32, TILE_FP64))
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-workloads", action="store_true", help="skip the droplet and flat-interface timings")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched-vs-sequential droplet sweep")
    ap.add_argument("--sweep-steps", type=int, default=2000)
    ap.add_argument("--cpu-n", type=int, default=2048)
    ap.add_argument("--cpu-steps", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
