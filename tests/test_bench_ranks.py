"""Host logic of the multi-GPU bench on CPU ranks (gloo, world size 2): the
job's time is its slowest rank's, the value counts every rank's builds, and
the reference arm prints only on rank 0."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local = [3.0, 5.0][rank]  # each rank's summed build seconds
    slowest = bench.ranks_max(local, world, "cpu")
    out[rank] = (slowest, bench.job_seconds_per_build(slowest, 4, world))
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_take_the_slowest_rank_and_count_all_builds():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        slowest, value = out[rank]
        assert slowest == 5.0
        assert value == pytest.approx(5.0 / 8)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.ranks_max(2.5, 1, "cpu") == 2.5
    assert bench.job_seconds_per_build(6.0, 3, 1) == pytest.approx(2.0)


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_traffic_reported_only_for_the_sources_it_was_measured_on(monkeypatch):
    """The roofline's DRAM traffic is an ncu counter of one kernel build: a
    recorded value whose source hash no longer matches reads as null."""
    import bench

    sha = bench.kernel_sources_sha256()
    monkeypatch.setattr(bench, "TRAFFIC", {("w", "p"): (sha, 1.5e9), ("w", "q"): ("0" * 64, 2.5e9)})
    assert bench.measured_traffic("w", "p") == 1.5e9
    assert bench.measured_traffic("w", "q") is None  # kernel changed since the capture
    assert bench.measured_traffic("other", "p") is None


def test_traffic_hash_ignores_comments_but_not_code():
    import bench

    src = "int f(int x) {  // doubles x\n  /* a\n block */ return 2 * x;\n}\n"
    assert bench.code_of(src) == bench.code_of("int f(int x) {\n\n   return 2 * x;\n}")
    assert bench.code_of(src) != bench.code_of(src.replace("2 * x", "3 * x"))


def test_clock_samples_summarised_with_every_active_throttle_reason():
    import bench

    lines = [
        "2070, 2070, 512.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "1965, 2070, 1398.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "[N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "2070, 2070, 880.1, 0x0000000000000008, Active, Not Active, Not Active, Not Active\n",
        "garbled line\n",
    ]
    c = bench.summarise_clocks(lines)
    assert c["samples"] == 4
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["power_w_max"] == 1398.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.summarise_clocks(["garbled\n"]) is None
