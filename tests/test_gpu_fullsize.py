"""Full-size parity: the dense tall 1,000,000 x 2000 problem (rank 1800, cond
1e6) in the configuration the benchmark times (tensor-core sketch, double-float
and FP64 passes), and the sparse 10^4 x 10^6 Tikhonov problem (2000 nonzeros
per row, lambda = 1e-3).  The oracle cannot run LSRN at these sizes, so it
checks what it can compute directly:
  * sketch entries A~[k, j] = sum_i G[k, i] A[i, j], drawn one by one from the
    oracle's generator and an FP64 dot product over the 10^6 rows;
  * x against x* = V Sigma^-1 U^T b from the generator's planted factors
    (section 2.1), and the normal-equation residual ||A^T r|| / (||A|| ||r||);
  * for the sparse case, x against the ridge closed form A^T (A A^T + lam^2 I)^-1 b
    (section 5), formed from the sparse A A^T and a Cholesky factorisation."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


@pytest.fixture(scope="module")
def c2():
    P = W.c2_problem(seed=0, device="cuda")
    return P, np.ascontiguousarray(P.A.cpu().numpy()), P.b.cpu().numpy()


@pytest.mark.parametrize("iter_mode", ["x2", "f64"])
def test_dense_tall_full_size(c2, iter_mode):
    P, A_host, b = c2
    m, n = P.A.shape
    mode = L.LSRN_ITER_F32X2 if iter_mode == "x2" else L.LSRN_ITER_F64
    opt = L.default_options(seed=1234, sketch_mode=L.LSRN_SKETCH_TC_SLICED, iter_mode=mode)
    plan = L.lsrn_plan(P.A, opt)
    try:
        L.lsrn_sketch(plan)
        S = L.lsrn_plan_get_sketch(plan)
        x, info = L.lsrn_solve_lsqr(plan, P.b)
    finally:
        plan.close()
    assert S.shape == (math.ceil(2 * n), n)
    assert info["rank"] == 1800
    # sampled sketch entries, computed by the oracle one at a time
    rng = np.random.Generator(np.random.PCG64(7))
    for k, j in zip(rng.integers(0, S.shape[0], 4), rng.integers(0, n, 4)):
        g = O.sketch_block(1234, 0, int(k), m, 1)[:, 0]          # G[k, :] = Gamma[:, k]
        col = A_host[:, int(j)]
        ref = float(np.dot(g, col))
        scale = float(np.dot(np.abs(g), np.abs(col)))
        assert abs(S[k, j] - ref) <= 1e-13 * scale
    # solution against the planted x*
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, b)
    xh = x.cpu().numpy()
    assert O.rel_err(xh, xs) <= 1e-10
    # normal-equation residual in double-double on the host (sigma_max = ||A|| = 1)
    r = O.dd_residual(A_host, b, xh)
    assert np.linalg.norm(O.dd_atr(A_host, r)) / np.linalg.norm(r) <= 1e-12


def test_dense_tall_full_size_cs(c2):
    """Algorithm 3 (Chebyshev semi-iterative) at full size in the benchmark's
    double-float mode: x against the planted x* and the normal equations."""
    P, A_host, b = c2
    opt = L.default_options(seed=1234, sketch_mode=L.LSRN_SKETCH_TC_SLICED,
                            iter_mode=L.LSRN_ITER_F32X2)
    plan = L.lsrn_plan(P.A, opt)
    try:
        x, info = L.lsrn_solve_cs(plan, P.b)
    finally:
        plan.close()
    assert info["rank"] == 1800 and info["sigma_L"] > 0.0
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, b)
    xh = x.cpu().numpy()
    assert O.rel_err(xh, xs) <= 1e-10
    r = O.dd_residual(A_host, b, xh)
    assert np.linalg.norm(O.dd_atr(A_host, r)) / np.linalg.norm(r) <= 1e-12


@pytest.fixture(scope="module")
def c3():
    A, b = W.c3_problem(seed=0)
    return A, b


def test_sparse_fat_ridge_full_size(c3):
    import scipy.sparse as sp
    A, b = c3
    lam = 1e-3
    csr = (A.m, A.n, torch.from_numpy(A.row_ptr).to("cuda"), torch.from_numpy(A.col_idx).to("cuda"),
           torch.from_numpy(A.values).to("cuda"))
    plan = L.lsrn_plan(None, L.default_options(seed=3, lambda_=lam), csr=csr)
    try:
        bt = torch.from_numpy(b).to("cuda")
        x_lsqr, info = L.lsrn_solve_lsqr(plan, bt)
        x_cs, _ = L.lsrn_solve_cs(plan, bt)
    finally:
        plan.close()
    assert info["tall"] == 0 and info["rank"] == A.m
    As = sp.csr_matrix((A.values, A.col_idx, A.row_ptr), shape=(A.m, A.n))
    ref = O.ridge_closed_form(As, b, lam)
    assert O.rel_err(x_lsqr.cpu().numpy(), ref) <= 1e-10
    assert O.rel_err(x_cs.cpu().numpy(), ref) <= 1e-10


def test_sparse_fat_ridge_full_size_f32_values():
    """The same 10^4 x 10^6 shape with FP32 values (the oracle uses the rounded
    values), with the QR preconditioner N = R^-1 of the full-rank augmented
    matrix: LSQR against the ridge closed form."""
    import scipy.sparse as sp
    A, b = W.c3_problem(seed=1, dtype=np.float32)
    lam = 1e-3
    csr = (A.m, A.n, torch.from_numpy(A.row_ptr).to("cuda"), torch.from_numpy(A.col_idx).to("cuda"),
           torch.from_numpy(A.values).to("cuda"))
    plan = L.lsrn_plan(None, L.default_options(seed=4, lambda_=lam, precond_mode=L.LSRN_PRECOND_QR),
                       csr=csr)
    try:
        x, info = L.lsrn_solve_lsqr(plan, torch.from_numpy(b).to("cuda"))
    finally:
        plan.close()
    assert info["tall"] == 0 and info["rank"] == A.m
    As = sp.csr_matrix((A.values.astype(np.float64), A.col_idx, A.row_ptr), shape=(A.m, A.n))
    ref = O.ridge_closed_form(As, b, lam)
    assert O.rel_err(x.cpu().numpy(), ref) <= 1e-10
