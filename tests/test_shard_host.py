"""Host side of the row-sharded path, without a GPU: the row partition, and
the exchange contract (rank-major allgather, then a sum in rank order) over a
world-size-2 gloo process group.  The per-shard quantities are the oracle's:
each rank sketches its block of rows with G drawn at the block's global row
indices, and the gathered partial sketches must add up to the sketch of the
whole matrix; likewise the partial A_p^T u_p add up to A^T u."""
import math
import os
import socket

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


@pytest.mark.parametrize("m,world", [(10, 1), (10, 3), (1000, 8), (7, 7), (1_000_003, 8)])
def test_shard_rows_partition(m, world):
    parts = [L.shard_rows(m, world, r) for r in range(world)]
    assert parts[0][0] == 0
    for (o1, c1), (o2, _) in zip(parts, parts[1:]):
        assert o2 == o1 + c1
    assert sum(c for _, c in parts) == m
    assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        L.shard_rows(3, 4, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, n, seed = 301, 13, 9
        s = math.ceil(2 * n)
        A = np.random.Generator(np.random.PCG64(1)).standard_normal((m, n))
        u = np.random.Generator(np.random.PCG64(2)).standard_normal(m)
        off, cnt = L.shard_rows(m, world, rank)
        Gp = O.sketch_block(seed, off, 0, cnt, s)               # rows off .. off+cnt of Gamma
        part = np.concatenate([(Gp.T @ A[off:off + cnt]).ravel(), A[off:off + cnt].T @ u[off:off + cnt]])
        recv = torch.empty(world * part.size, dtype=torch.float64)
        dist.all_gather_into_tensor(recv, torch.from_numpy(part))
        blocks = recv.numpy().reshape(world, part.size)
        total = blocks[0].copy()
        for p in range(1, world):                               # rank order
            total += blocks[p]
        full_sketch = (O.sketch_block(seed, 0, 0, m, s).T @ A).ravel()
        ok = (np.allclose(total[:s * n], full_sketch, rtol=0, atol=1e-12 * np.abs(full_sketch).max())
              and np.allclose(total[s * n:], A.T @ u, rtol=0, atol=1e-12 * np.abs(A.T @ u).max()))
        q.put((rank, bool(ok), total.tobytes()))
    finally:
        dist.destroy_process_group()


def test_gloo_world2_gathered_partials_sum_to_the_whole():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert all(ok for _, ok, _ in res)
    assert res[0][2] == res[1][2]          # both ranks hold the same bits
