"""Row-sharded solve (section 4.4): A split by rows over shards, one plan per
shard, exchanges through an allgather callback.  Here the shards are host
threads sharing one GPU: each has its own plan and stream, and the callback
meets the other threads at a host barrier, so no kernel ever waits for another
shard's kernel.  Checked: every shard returns the same x, bit for bit; x
matches the oracle's min-length (or ridge) solution at the parity tolerance
and the unsharded solve closely; a failing exchange is reported as
LSRN_ERR_COMM; bad shard descriptors are refused."""
import threading

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


class ThreadGather:
    """In-process allgather over `world` host threads (host staging)."""

    def __init__(self, world: int, fail_rank: int = -1):
        self.world = world
        self.slots = [None] * world
        self.barrier = threading.Barrier(world, timeout=120)
        self.fail_rank = fail_rank
        self.calls = 0

    def callback(self, rank: int):
        def fn(send_ptr, recv_ptr, count):
            if rank == self.fail_rank:
                self.barrier.abort()
                raise RuntimeError("planted exchange failure")
            self.calls += 1
            self.slots[rank] = L.device_view(send_ptr, count).cpu()
            self.barrier.wait()
            L.device_view(recv_ptr, count * self.world).copy_(torch.cat(self.slots))
            torch.cuda.synchronize()
            self.barrier.wait()          # nobody refills a slot before everyone has read
        return fn


def sharded_solve(A_host, b_host, world, solver="lsqr", csr=None, fail_rank=-1, **opts):
    shape = A_host.shape if csr is None else (csr.m, csr.n)
    by_cols = shape[0] < shape[1]                 # a fat A is split by columns
    m = shape[1] if by_cols else shape[0]         # the long side
    gather = ThreadGather(world, fail_rank)
    out = [None] * world

    def worker(rank):
        torch.cuda.set_device(0)
        off, cnt = L.shard_rows(m, world, rank)
        try:
            if csr is None and by_cols:
                A = torch.from_numpy(np.ascontiguousarray(A_host[:, off:off + cnt])).cuda()
                plan = L.lsrn_plan_sharded(A, L.default_options(**opts), rank, world, off, m,
                                           gather.callback(rank), by_columns=True)
            elif csr is None:
                A = torch.from_numpy(np.ascontiguousarray(A_host[off:off + cnt])).cuda()
                plan = L.lsrn_plan_sharded(A, L.default_options(**opts), rank, world, off, m,
                                           gather.callback(rank))
            else:
                rp = csr.row_ptr[off:off + cnt + 1] - csr.row_ptr[off]
                lo, hi = csr.row_ptr[off], csr.row_ptr[off + cnt]
                blk = (cnt, csr.n, torch.from_numpy(np.ascontiguousarray(rp)).cuda(),
                       torch.from_numpy(csr.col_idx[lo:hi].copy()).cuda(),
                       torch.from_numpy(csr.values[lo:hi].copy()).cuda())
                plan = L.lsrn_plan_sharded(None, L.default_options(**opts), rank, world, off, m,
                                           gather.callback(rank), csr=blk)
            bh = b_host if by_cols else b_host[off:off + cnt]     # fat: the whole b
            b = torch.from_numpy(np.ascontiguousarray(bh)).cuda()
            fn = L.lsrn_solve_lsqr if solver == "lsqr" else L.lsrn_solve_cs
            try:
                x, info = fn(plan, b)
                out[rank] = ("ok", x.cpu().numpy(), info)
            finally:
                plan.close()
        except L.LsrnError as e:
            out[rank] = ("err", e.status, None)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert all(not t.is_alive() for t in threads)
    return out


def _check_same_on_all_shards(out):
    assert all(o[0] == "ok" for o in out), out
    x0 = out[0][1]
    for o in out[1:]:
        assert np.array_equal(o[1], x0)
    return x0, out[0][2]


def _gather_blocks(out):
    """fat: each shard returns its block of x; all shards ran the same recurrences"""
    assert all(o[0] == "ok" for o in out), out
    for o in out[1:]:
        assert o[2]["iterations"] == out[0][2]["iterations"]
        assert o[2]["rank"] == out[0][2]["rank"]
    return np.concatenate([o[1] for o in out]), out[0][2]


@pytest.mark.parametrize("world,solver,lam", [(2, "lsqr", 0.0), (3, "cs", 0.0), (2, "lsqr", 0.2),
                                              (3, "cs", 0.2)])
def test_sharded_fat_by_columns(world, solver, lam):
    P = W.dense_householder(2600, 110, rank=100, cond=1e4, noise=0.0, seed=77)
    A = np.ascontiguousarray(P.A.T)                           # 110 x 2600
    b = np.random.Generator(np.random.PCG64(78)).standard_normal(110)
    out = sharded_solve(A, b, world, solver, seed=11, lambda_=lam)
    x, info = _gather_blocks(out)
    assert info["tall"] == 0 and info["m"] == 110
    ref = O.ridge_closed_form(A, b, lam) if lam > 0 else O.minlen_refined(A, b)[0]
    assert O.rel_err(x, ref) <= 1e-10
    x1, _ = L.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), solver=solver, seed=11,
                    lambda_=lam)
    assert O.rel_err(x, x1.cpu().numpy()) <= 1e-11


@pytest.mark.parametrize("world,solver", [(2, "lsqr"), (3, "cs")])
def test_sharded_dense_tall_matches_oracle_and_unsharded(world, solver):
    P = W.dense_householder(3001, 120, rank=110, cond=1e4, noise=1e-3, seed=71)
    out = sharded_solve(P.A, P.b, world, solver, seed=5)
    x, info = _check_same_on_all_shards(out)
    assert info["rank"] == 110 and info["m"] == 3001
    xs, _ = O.minlen_refined(P.A, P.b)
    assert O.rel_err(x, xs) <= 1e-10
    x1, _ = L.solve(torch.from_numpy(P.A).cuda(), torch.from_numpy(P.b).cuda(), solver=solver, seed=5)
    assert O.rel_err(x, x1.cpu().numpy()) <= 1e-11


def test_sharded_ridge_rows_on_shard_zero():
    P = W.dense_householder(2500, 90, rank=90, cond=1e3, noise=1e-2, seed=72)
    out = sharded_solve(P.A, P.b, 3, "lsqr", seed=6, lambda_=0.3)
    x, _ = _check_same_on_all_shards(out)
    assert O.rel_err(x, O.ridge_closed_form(P.A, P.b, 0.3)) <= 1e-10


def test_sharded_mixed_precision_tensor_core_sketch():
    P = W.dense_householder(40_000, 600, rank=560, cond=1e6, noise=1e-4, seed=73)
    out = sharded_solve(P.A, P.b, 2, "lsqr", seed=7, sketch_mode=L.LSRN_SKETCH_TC_SLICED,
                        iter_mode=L.LSRN_ITER_F32X2)
    x, info = _check_same_on_all_shards(out)
    assert info["rank"] == 560
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    assert O.rel_err(x, xs) <= 1e-10


def test_sharded_csr_tall():
    C = W.csr_random_density(6000, 70, 0.05, seed=74)
    b = np.random.Generator(np.random.PCG64(75)).standard_normal(6000)
    out = sharded_solve(None, b, 2, "lsqr", csr=C, seed=8)
    x, _ = _check_same_on_all_shards(out)
    xs, _ = O.minlen_refined(C.to_dense(), b)
    assert O.rel_err(x, xs) <= 1e-10


def test_failed_exchange_is_reported():
    P = W.dense_householder(2000, 50, rank=50, cond=1e2, noise=1e-3, seed=76)
    out = sharded_solve(P.A, P.b, 2, "lsqr", fail_rank=1, seed=9)
    assert [o[0] for o in out] == ["err", "err"]
    assert all(o[1] == L.LSRN_ERR_COMM for o in out)


def test_bad_shard_descriptors_are_refused():
    A = torch.zeros((100, 10), dtype=torch.float64, device="cuda")
    noop = lambda s, r, c: None
    for rank, world, off, mt, status in [(0, 0, 0, 100, L.LSRN_ERR_INVALID_ARG),
                                         (2, 2, 0, 200, L.LSRN_ERR_INVALID_ARG),
                                         (0, 2, 50, 120, L.LSRN_ERR_INVALID_ARG),
                                         (0, 2, 0, 5, L.LSRN_ERR_INVALID_ARG),
                                         (0, 2, 0, 101, None),
                                         (0, 1, 0, 100, None)]:
        if status is None:
            L.lsrn_plan_sharded(A, None, rank, world, off, mt, noop).close()
            continue
        with pytest.raises(L.LsrnError) as e:
            L.lsrn_plan_sharded(A, None, rank, world, off, mt, noop)
        assert e.value.status == status
    Af = torch.zeros((10, 100), dtype=torch.float64, device="cuda")   # rows of a fat A: not the long side
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_plan_sharded(Af, None, 0, 2, 0, 20, noop)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
    L.lsrn_plan_sharded(Af, None, 0, 2, 0, 300, noop, by_columns=True).close()
