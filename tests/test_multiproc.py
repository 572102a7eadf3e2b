"""Host side of the multi-process benchmark (replicas, one process per GPU) on CPU: two gloo ranks.

Images are independent, so the replicas exchange nothing on the data path; the process group serves the barrier and
the max-over-ranks timing, which these tests run with the gloo backend (no GPU)."""
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


def _rank_main(rank, world, port, values, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        m = bench.max_over_ranks(values[rank], world, device="cpu")
        out.put((rank, m, bench.job_rate(100, world, m)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks():
    world, port = 2, _free_port()
    values = [12.5, 40.0]  # ms of each rank's timed region
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, values, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the job rate counts both replicas' images over it
    assert [r[1] for r in results] == [40.0, 40.0]
    assert results[0][2] == pytest.approx(2 * 100 / 0.040)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_rate(50, 1, 250.0) == pytest.approx(200.0)
