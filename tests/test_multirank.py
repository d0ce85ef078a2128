"""The N > 1 host logic of bench.py on CPU: world_size-2 gloo process groups (one process
per rank, as torchrun launches them). Each rank trains its own replica, so the job time is
the maximum over ranks and the whole-job rate counts every rank's units; the reference arm
runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        got_ws, got_rank, got_local = bench.dist_env()
        job = bench.job_time_ms(100.0 * (rank + 1), ws)       # rank r took (r + 1) x 100 ms
        rate = bench.whole_job_rate(50, ws, job)
        out[rank] = (got_ws, got_rank, got_local, job, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_rate_counts_all_ranks():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    for r in range(ws):
        got_ws, got_rank, got_local, job, rate = out[r]
        assert (got_ws, got_rank, got_local) == (ws, r, r)
        assert job == 200.0                     # the slower rank ends the job
        assert rate == pytest.approx(50 * ws / 0.2)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.job_time_ms(123.0, 1) == 123.0
    assert bench.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(trees=1000, steps=1, warmup=1, ref_sample_trees=1)
    assert bench.run_reference(args) == 0     # returns before any work


def test_recorded_traffic_needs_the_same_kernel_source_and_variant(tmp_path, monkeypatch):
    """bench.py reports the ncu DRAM traffic of the histogram kernel only from a capture
    taken on the current kernel source and on the selected --hist-kernel variant."""
    import bench
    h = bench.hist_source_hash()
    (tmp_path / "hist_kernel_traffic_red.txt").write_text(
        f"# comment\nsource_sha256_16 {h}\nkernel_variant red\ndram_bytes_per_row 321.4\n")
    (tmp_path / "hist_kernel_traffic_int.txt").write_text(
        "source_sha256_16 0000000000000000\nkernel_variant int\ndram_bytes_per_row 285.1\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "hist_kernel_traffic_{}.txt"))
    assert bench.recorded_traffic_per_row("red") == 321.4
    assert bench.recorded_traffic_per_row("int") is None      # taken on another source
    assert bench.recorded_traffic_per_row("lane") is None     # no capture for the variant
    (tmp_path / "hist_kernel_traffic_lane.txt").write_text(
        f"source_sha256_16 {h}\nkernel_variant lane\ndram_bytes_per_row 200.0\n")
    assert bench.recorded_traffic_per_row("lane") is None     # the red kernel's source hash
    (tmp_path / "hist_kernel_traffic_lane.txt").write_text(
        f"source_sha256_16 {bench.hist_source_hash('lane')}\nkernel_variant lane\ndram_bytes_per_row 200.0\n")
    assert bench.recorded_traffic_per_row("lane") == 200.0
