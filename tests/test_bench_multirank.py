"""The benchmark's multi-rank host logic on CPU with the gloo backend
(world size 2): the timed region is the maximum over ranks, the job value
counts every rank's problems, and under the reference arm only rank 0 works.
Each rank solves an independent problem, so no data-path collective exists to
test beyond the timing reduction."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # ranks finish at different times; everyone reports the slowest
        elapsed = 100.0 + 50.0 * rank
        worst = bench.max_over_ranks(elapsed, dist, "cpu")
        value = bench.job_throughput(world, 3, worst)
        # the reference arm: ranks other than 0 return at once without output
        ref_rc = bench.run_reference(bench.parse([])) if rank != 0 else 0
        out.put((rank, worst, value, ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, worst, value, ref_rc in res:
        assert worst == 150.0
        assert value == pytest.approx(2 * 3 / 0.150)
        assert ref_rc == 0


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(1, 4, 2000.0) == pytest.approx(2.0)
