"""Single-pass BF16 tensor-core sketch (LSRN_SKETCH_BF16) and the AUTO mode.

The BF16 sketch rounds G and A to bf16 once and accumulates in FP32 on the
tensor cores (per 2048 rows, FP64 beyond), so each entry of A~ = G^T-style
contraction is off by at most ~2^-8 of sum |g| |a| (two bf16 roundings of
2^-9 each, plus the FP32 accumulation).  Parity is checked entry by entry
against the oracle's G^T A under that bound, on shapes spanning several
128 x 256 tiles with ragged edges, several row segments, K splits and column
scales far outside FP32's range (per-column exponents).  Solves: a
well-conditioned full-rank problem keeps the BF16 preconditioner under AUTO
and still reaches the parity tolerance (the iterations use the FP64 A); a
rank-deficient kappa = 1e6 problem makes AUTO switch to the exact sketch."""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")

BF16_BOUND = 2.0 ** -7          # per entry, relative to sum_l |G[k, l]| |X[l, j]|


def _oracle_sketch_and_scale(A, seed):
    m, n = A.shape
    if m >= n:
        G = O.sketch_block(seed, 0, 0, m, math.ceil(2 * n))          # Gamma (m x s)
        return G.T @ A, np.abs(G).T @ np.abs(A)
    G = O.sketch_block(seed, 0, 0, n, math.ceil(2 * m))              # Gamma (n x s)
    return (A @ G).T, (np.abs(A) @ np.abs(G)).T


@pytest.mark.parametrize("m,n,seg,scaled", [(3001, 300, None, False), (301, 2999, None, False),
                                            (5000, 257, "1024", False), (2500, 130, None, True)])
def test_bf16_sketch_entrywise_bound(m, n, seg, scaled):
    rng = np.random.Generator(np.random.PCG64(m + 7 * n))
    A = rng.standard_normal((m, n))
    if scaled:                                   # columns at 2^-300 .. 2^300
        A *= np.exp2(rng.integers(-300, 301, size=n)).astype(np.float64)[None, :]
    if seg:
        os.environ["LSRN_TC_SEGMENT_ROWS"] = seg
    try:
        plan = L.lsrn_plan(torch.from_numpy(A).cuda(),
                           L.default_options(seed=13, sketch_mode=L.LSRN_SKETCH_BF16))
        L.lsrn_sketch(plan)
        S = L.lsrn_plan_get_sketch(plan)
        plan.close()
    finally:
        os.environ.pop("LSRN_TC_SEGMENT_ROWS", None)
    ref, scale = _oracle_sketch_and_scale(A, 13)
    assert S.shape == ref.shape and np.all(np.isfinite(S))
    ratio = np.abs(S - ref) / np.maximum(scale, 1e-300)
    assert ratio.max() <= BF16_BOUND
    rel = np.linalg.norm((S - ref) / np.maximum(scale, 1e-300)) / math.sqrt(S.size)
    assert 1e-5 < rel < 5e-3                    # bf16 error, neither exact nor garbage


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_auto_keeps_bf16_for_a_well_conditioned_problem(solver):
    P = W.dense_householder(20_000, 300, rank=300, cond=10.0, noise=1e-3, seed=81)
    x, info = L.solve(torch.from_numpy(P.A).cuda(), torch.from_numpy(P.b).cuda(), solver=solver,
                      seed=3, sketch_mode=L.LSRN_SKETCH_AUTO)
    assert info["sketch_used"] == L.LSRN_SKETCH_BF16 and info["sketch_escalated"] == 0
    xs, _ = O.minlen_refined(P.A, P.b)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10


def test_bf16_fat_well_conditioned():
    P = W.dense_householder(6000, 250, rank=250, cond=8.0, noise=0.0, seed=82)
    A = np.ascontiguousarray(P.A.T)                       # 250 x 6000, m < n
    b = np.random.Generator(np.random.PCG64(83)).standard_normal(250)
    x, info = L.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), solver="lsqr",
                      seed=4, sketch_mode=L.LSRN_SKETCH_BF16)
    assert info["tall"] == 0 and info["sketch_used"] == L.LSRN_SKETCH_BF16
    xs, _ = O.minlen_refined(A, b)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_auto_escalates_on_rank_deficient_ill_conditioned(solver):
    P = W.c1_problem(0)                                   # 2000 x 100, rank 80, cond 1e6
    x, info = L.solve(torch.from_numpy(P.A).cuda(), torch.from_numpy(P.b).cuda(), solver=solver,
                      seed=5, sketch_mode=L.LSRN_SKETCH_AUTO)
    assert info["sketch_escalated"] == 1 and info["sketch_used"] == L.LSRN_SKETCH_TC_SLICED
    assert info["rank"] == 80
    xs, _ = O.minlen_refined(P.A, P.b)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10


def test_auto_on_csr_uses_the_fp64_sketch():
    C = W.csr_random_density(3000, 60, 0.05, seed=84)
    b = np.random.Generator(np.random.PCG64(85)).standard_normal(3000)
    csr = (C.m, C.n, torch.from_numpy(C.row_ptr).cuda(), torch.from_numpy(C.col_idx).cuda(),
           torch.from_numpy(C.values).cuda())
    x, info = L.solve(None, torch.from_numpy(b).cuda(), csr=csr, seed=6,
                      sketch_mode=L.LSRN_SKETCH_AUTO)
    assert info["sketch_used"] == L.LSRN_SKETCH_F64
    xs, _ = O.minlen_refined(C.to_dense(), b)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10
