"""Host logic of bench.py on CPU: in multi-rank mode two gloo ranks (replicas
only, no data-path collective) agree on the slowest rank's time, and the
whole-job value counts every rank's samples; the roofline helpers pick the
dominant kernel and compute its fraction of the peak."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
        got = bench.max_over_ranks(ms, world, "cpu")
        value = bench.whole_job_value(1_000_000, got, world)
        q.put((rank, got, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, got, value in res:
        assert got == 15.0
        # 2 ranks x 1e6 samples in 15 ms
        assert value == pytest.approx(2 * 1e6 / 15e-3 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_value(10**6, 1.0, 1) == pytest.approx(1000.0)


def test_dominant_roofline_picks_the_largest_share():
    """The roofline reports the kernel (as ncu names it) with the largest total
    time over the passes it runs, at its mean launch time, against the measured
    (or fallback) HBM peak; its traffic comes from the ncu table by name."""
    import bench
    names = ["k<0, 1>", "k<1, 4>", "k<0, 2>", "k<1, 4>", "k<0, 3>"]
    pass_ms = [0.060, 0.096, 0.093, 0.094, 0.070]
    r = bench._dominant_roofline(pass_ms, names, 268_435_456, {"k<1, 4>": 2.0e8})
    peak, _ = bench._peaks()
    assert r["kernel"] == "k<1, 4>"                       # 0.190 ms against 0.093 at most for the others
    assert abs(r["avg_launch_ms"] - 0.095) < 1e-12
    assert abs(r["share"] - 0.190 / sum(pass_ms)) < 1e-12
    assert abs(r["achieved"] - 268_435_456 / 0.095e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12 and r["peak"] == peak
    assert r["traffic"] == 2.0e8 and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # a kernel the ncu table does not list reports no traffic
    assert bench._dominant_roofline([1.0, 2.0], ["a", "b"], 1, None)["traffic"] is None


def test_pass_kernel_table_covers_every_schedule():
    """Every (precision, pass count) the main workload can run has one kernel
    name per pass, and the FP32 ones are the line-pair kernel's instantiations
    whose ncu traffic is recorded."""
    import bench
    for (prec, npass), names in bench.PASS_KERNELS.items():
        assert len(names) == npass, (prec, npass)
        if prec == "fp32":
            assert all(n in bench.NCU_TRAFFIC for n in names)
