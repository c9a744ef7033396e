"""The benchmark's multi-process arithmetic on CPU: two gloo ranks (one
process per GPU in the real run, replicas with no data-path collective)
agree on the slowest rank's time, and the job's throughput counts every
rank's points against that time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [12.5, 40.0][rank]            # this rank's mean step time, ms
        ms = bench.max_over_ranks(mine, dist, "cpu")
        out[rank] = (ms, bench.job_points_per_s(world, 1000, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 40.0
    assert value == pytest.approx(2 * 1000 / 0.040)


def test_single_process_keeps_its_time():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(17.0) == 17.0
    assert bench.job_points_per_s(1, 4096, 2.0) == pytest.approx(4096 / 0.002)


def test_class_roofline_arithmetic():
    """Per-class roofline figures from a class's algorithmic bytes / flops
    and its time: HBM-bound classes in GB/s against the copy peak, the
    others in TFLOP/s against the derived FP32 peak; no time, no figure."""
    sys.path.insert(0, ROOT)
    import bench

    peaks = {"hbm": 6800.0, "sm_mhz": 2070.0}
    r = bench.class_roofline("schur", {"ms": 2.0, "bytes": 6.8e9, "flops": 0.0, "launches": 5}, peaks, "mixed")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3400.0) and r["frac"] == pytest.approx(0.5)
    r = bench.class_roofline("id", {"ms": 10.0, "bytes": 0.0, "flops": 1e11, "launches": 9}, peaks, "mixed")
    pk = bench.alu_peak_tflops("mixed", 2070.0)
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(10.0) and r["frac"] == pytest.approx(10.0 / pk)
    assert bench.class_roofline("elim", {"ms": 0.0, "bytes": 0.0, "flops": 0.0, "launches": 0}, peaks, "mixed") is None
