"""Matrix-free operator (lsrn_plan_operator): A enters only through products
(the paper applies A and A^T and never forms anything else of A), given as
callbacks on blocks of vectors.  The sketch is built from blocks of G's columns
(A^T G^T or A G), the iterations from one product with A and one with A^T each.
Checked against the oracle's min-length / ridge solutions and against the same
problem as a stored matrix, for dense and sparse operators, tall and fat."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _dense_op(A):
    At = torch.from_numpy(A).cuda()

    def matmat(x, y):          # x: (k, n) rows = columns of the block; y: (k, m)
        y.copy_((At @ x.T).T)

    def rmatmat(y, x):
        x.copy_((At.T @ y.T).T)
    return matmat, rmatmat


def _sparse_op(C):
    S = torch.sparse_csr_tensor(torch.from_numpy(C.row_ptr), torch.from_numpy(C.col_idx.astype(np.int64)),
                                torch.from_numpy(C.values), size=(C.m, C.n)).cuda()
    St = S.to_dense().T.to_sparse_csr()

    def matmat(x, y):
        y.copy_((S @ x.T.contiguous()).T)

    def rmatmat(y, x):
        x.copy_((St @ y.T.contiguous()).T)
    return matmat, rmatmat


@pytest.mark.parametrize("shape,solver,lam", [((4000, 150), "lsqr", 0.0), ((4000, 150), "cs", 0.0),
                                              ((120, 3000), "lsqr", 0.0), ((2500, 90), "cs", 0.3),
                                              ((90, 2500), "lsqr", 0.2)])
def test_dense_operator(shape, solver, lam):
    m, n = shape
    q = min(m, n)
    P = W.dense_householder(max(m, n), q, rank=q, cond=1e2, noise=1e-3, seed=161)
    A = P.A if m >= n else np.ascontiguousarray(P.A.T)
    b = P.b if m >= n else np.random.Generator(np.random.PCG64(162)).standard_normal(m)
    mm, rm = _dense_op(A)
    plan = L.lsrn_plan_operator(m, n, mm, rm, L.default_options(seed=8, lambda_=lam))
    try:
        fn = L.lsrn_solve_lsqr if solver == "lsqr" else L.lsrn_solve_cs
        x, info = fn(plan, torch.from_numpy(b).cuda())
    finally:
        plan.close()
    assert info["refine_steps"] == 0 and info["rank"] == q
    ref = O.ridge_closed_form(A, b, lam) if lam > 0 else O.minlen_refined(A, b)[0]
    assert O.rel_err(x.cpu().numpy(), ref) <= 1e-10
    xd, _ = L.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), solver=solver, seed=8,
                    lambda_=lam, refine_max=0)
    assert O.rel_err(x.cpu().numpy(), xd.cpu().numpy()) <= 1e-11


def test_rank_deficient_operator_matches_stored_matrix():
    P = W.dense_householder(3000, 120, rank=100, cond=1e4, noise=1e-3, seed=163)
    mm, rm = _dense_op(P.A)
    plan = L.lsrn_plan_operator(3000, 120, mm, rm, L.default_options(seed=9))
    try:
        x, info = L.lsrn_solve_lsqr(plan, torch.from_numpy(P.b).cuda())
    finally:
        plan.close()
    assert info["rank"] == 100
    xd, _ = L.solve(torch.from_numpy(P.A).cuda(), torch.from_numpy(P.b).cuda(), seed=9, refine_max=0)
    assert O.rel_err(x.cpu().numpy(), xd.cpu().numpy()) <= 1e-9


def test_sparse_operator():
    C = W.csr_sprandn(20_000, 80, 0.02, seed=164)
    b = np.random.Generator(np.random.PCG64(165)).standard_normal(C.m)
    mm, rm = _sparse_op(C)
    plan = L.lsrn_plan_operator(C.m, C.n, mm, rm, L.default_options(seed=10))
    try:
        x, _ = L.lsrn_solve_lsqr(plan, torch.from_numpy(b).cuda())
    finally:
        plan.close()
    assert O.rel_err(x.cpu().numpy(), O.minlen_refined(C.to_dense(), b)[0]) <= 1e-10


def test_operator_failures():
    import ctypes
    h = ctypes.c_void_p()
    assert L.load_library().lsrn_plan_operator(None, None, None, ctypes.byref(h)) == L.LSRN_ERR_INVALID_ARG
    op = L.lsrn_operator(m=50, n=5)                                  # no callbacks
    assert L.load_library().lsrn_plan_operator(ctypes.byref(op), None, None,
                                               ctypes.byref(h)) == L.LSRN_ERR_INVALID_ARG
    mm, rm = _dense_op(np.ones((50, 5)))

    def bad(x, y):
        raise RuntimeError("planted product failure")
    plan = L.lsrn_plan_operator(50, 5, mm, bad, L.default_options(seed=1))
    try:
        with pytest.raises(L.LsrnError) as e:
            L.lsrn_sketch(plan)
        assert e.value.status == L.LSRN_ERR_COMM
    finally:
        plan.close()
