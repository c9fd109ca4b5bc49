"""CPU checks of bench.py: the reference arm (the oracle timed on the host cores) prints the JSON
line of the bench contract, alone and as rank 0 of two torchrun ranks; the step time of a
multi-rank job is the largest over the ranks (two gloo ranks); and the roofline entries scale the
measured per-subdomain DRAM traffic by the launch's subdomains and divide the algorithmic work by the
measured launch time."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "config", "e2e",
                "cpu_baseline"):
        assert key in line, key
    assert line["higher_is_better"] is False and line["unit"] == "s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_roofline_entry_arithmetic():
    import bench
    # 3 launches, 6 ms and 6e12 flops in all: 2e12 flops per launch / 2 ms = 1000 TFLOP/s
    e = bench.roofline_entry("eig_orthogonalisation", 3, 6.0, 6e12, 6780.0, subdomains=256)
    assert e["bound"] == "alu" and e["dtype"] == "f32x2"
    assert e["achieved"] == pytest.approx(1000.0)
    assert e["frac"] == pytest.approx(1000.0 / bench.FP32X2_PEAK_TFLOPS_DERIVED)
    # the tensor-core double-float kernels: the measured BF16 peak over the 28 digit-pair products
    e = bench.roofline_entry("eig_triangular_solves", 3, 6.0, 6e12, 6780.0, subdomains=256)
    assert e["bound"] == "tensor" and e["traffic"] is None
    bf16 = bench.measured_peaks().get(bench.BF16_PEAK_KEY)
    if bf16:
        assert e["peak"] == pytest.approx(bf16 / 28) and e["frac"] == pytest.approx(1000.0 / (bf16 / 28))
    # the plain form's kernels use the FP64 peak
    e = bench.roofline_entry("coarse_lu", 1, 1.0, 1e9, 6780.0, fp32=False, subdomains=256)
    assert e["traffic"] is None and e["peak"] == bench.FP64_PEAK_TFLOPS_NOMINAL
    # the apply's local solves are HBM bound: 1e9 bytes per launch / 0.5 ms against the measured copy rate
    e = bench.roofline_entry("apply_local_solves", 2, 1.0, 2e9, 6780.0)
    assert e["bound"] == "hbm" and e["achieved"] == pytest.approx(2000.0)
    assert e["frac"] == pytest.approx(2000.0 / 6780.0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_over_ranks_worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, bench.max_over_ranks([3.5, 7.25][rank], world)))
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_largest_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_max_over_ranks_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 7.25, 1: 7.25}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5


def test_reference_arm_under_torchrun_prints_once():
    # two ranks on one node: rank 0 times the oracle and prints the line, rank 1 exits 0 without work
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
                        os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0", "--workload", "c3_small"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_forced_options_only_when_given():
    import argparse
    import bench
    a = argparse.Namespace(local_solve_kernel=0, eig_block_size=0)
    assert bench.forced_options(a, "fp32") == {} and bench.forced_options(a, "fp64") == {}
    a = argparse.Namespace(local_solve_kernel=3000, eig_block_size=18)
    assert bench.forced_options(a, "fp32") == {"local_solve_kernel": 3000, "eig_block_size": 18}
    assert bench.forced_options(a, "fp64") == {"eig_block_size": 18}  # the streaming kernel is FP32/BF16 only
