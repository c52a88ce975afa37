"""bench.py's multi-rank host logic on CPU: two gloo ranks agree on the
slowest rank's time and on the whole-job throughput, and the reference arm
does its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    out[rank] = (t, bench.whole_job_mlups(world, 4096 * 4096, 100, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.0
    assert abs(out[0][1] - 2 * 4096 * 4096 * 100 / 2.0 / 1e6) < 1e-6


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, nx, ny = 3, 3, 4096, 4096
    assert bench.run_reference(A) == 0
    assert capsys.readouterr().out == ""


def test_traffic_figure_is_used_only_for_the_profiled_kernel():
    """The committed ncu traffic applies to the kernel it names and only while
    the kernel's sources (kernel file and the header it compiles) hash to the
    value recorded beside it."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    h = hashlib.sha256()
    for name in ("lbm_step_kernels.cuh", "lbm_step_f32.cu", "lbm_step_f64.cu", "lbm_step.cu", "lbm_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1412_7228_gb300", "csrc", name), "rb").read())
    sha = h.hexdigest()[:16]
    assert bench.kernel_sources_sha() == sha
    path = os.path.join(ROOT, "profiles", "step_fp32_4096_traffic.txt")
    kv = dict(l.strip().split("=", 1) for l in open(path) if "=" in l and not l.startswith("#"))
    got = bench.kernel_traffic("fp32", kv["kernel"])
    if kv["kernel_sources_sha256_16"] == sha:
        assert got == float(kv["bytes_per_update"]) and 72.0 <= got < 80.0
    else:
        assert got is None
    assert bench.kernel_traffic("fp32", "lbm::some_other_kernel") is None


def test_fp64_roofline_and_cpu_model_records(tmp_path):
    """The FP64 roofline divides the oracle's operation count per update
    times the update rate by the measured FP64 peak; the ncu figures of the
    FP64 kernel are used only for the kernel they name; the CPU model is
    read from x86 and Arm cpuinfo alike."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    ops = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_op_count.json")))
    ops = ops["counts"]["carnahan_starling"]["flops_per_update"]
    assert bench.oracle_flops_per_update() == ops
    r = bench.fp64_roofline(2000.0, 1.25e12)
    assert r["bound"] == "alu" and r["peak_kind"] == "measured" and r["unit"] == "GFLOP/s"
    assert abs(r["achieved"] - ops * 2000.0e6 / 1e9) < 1e-9 and abs(r["frac"] - r["achieved"] / 1250.0) < 1e-12
    assert bench.fp64_roofline(2000.0, None) is None
    assert bench.fp64_pipe_profile("lbm::another_kernel") is None
    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nmodel name\t: Some CPU @ 2.0GHz\n")
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n")
    assert bench.cpu_model(str(x86)) == "Some CPU @ 2.0GHz"
    assert bench.cpu_model(str(arm)) == "Arm Neoverse V2 (part 0xd4f)"


def test_graph_use_reports_the_replayed_steps():
    """lbm_step(n) with graphs replays 32-, 16-, 8-, 4- and 2-step graphs for
    every even part of n and launches an odd last step plainly; the bench line
    reports that split."""
    import bench
    assert bench.graph_use(20) == {"graphs": True, "graph_steps": 20, "plain_launch_steps": 0}
    assert bench.graph_use(2000) == {"graphs": True, "graph_steps": 2000, "plain_launch_steps": 0}
    assert bench.graph_use(37) == {"graphs": True, "graph_steps": 36, "plain_launch_steps": 1}
    assert bench.graph_use(1) == {"graphs": False, "graph_steps": 0, "plain_launch_steps": 1}
