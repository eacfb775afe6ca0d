"""Double-float Jacobi pre-sweeps (LSRN_SVD_DF, 1024 < q <= 4096).

The early sweeps run on a double-float copy of R with the rotations
accumulated into P; Y = P R in FP64 then goes through the FP64 sweeps.  The
preconditioner must be the FP64 path's: the same rank, the singular values of
the sketch (against LAPACK's SVD of the same sketch, a library routine, and
against the FP64-only sweeps), Lemma 4.3 for A N, and the solve's accuracy
against x* from the planted factors."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _precond(A, mode, seed):
    plan = L.lsrn_plan(_dev(A), L.default_options(seed=seed, svd_mode=mode))
    try:
        L.lsrn_sketch(plan)
        S = L.lsrn_plan_get_sketch(plan)
        r = L.lsrn_precond(plan)
        N, sig = L.lsrn_plan_get_precond(plan)
    finally:
        plan.close()
    return S, r, N, sig


@pytest.mark.parametrize("n", [1100, 2000, 2500])
def test_df_presweeps_give_the_fp64_preconditioner(n):
    m = 3 * n + 11
    rank = n - 40
    P = W.dense_householder(m, n, rank, 1e6, 1e-4, seed=n % 89)
    S, r, N, sig = _precond(P.A, L.LSRN_SVD_DF, 5)
    S64, r64, N64, sig64 = _precond(P.A, L.LSRN_SVD_F64, 5)
    assert np.array_equal(S, S64)
    assert r == r64 == rank
    ref = np.linalg.svd(S, compute_uv=False)
    # backward-stable to FP64: |sigma - sigma_ref| within 1e-13 sigma_1 plus 1e-10 relative
    bound = 1e-13 * ref[0] + 1e-10 * ref[:r]
    assert np.all(np.abs(sig - ref[:r]) <= bound)
    assert np.all(np.abs(sig - sig64) <= bound)
    # the numerical rank's cut: the discarded singular values sit far below it
    rcond = max(S.shape) * 2.0**-53
    assert sig[-1] > 1e3 * rcond * sig[0]
    # Lemma 4.3: sigma(A N) = 1 / sigma(G U); both N give the same spectrum
    got = np.sort(np.linalg.svd(P.A @ N, compute_uv=False))
    got64 = np.sort(np.linalg.svd(P.A @ N64, compute_uv=False))
    assert np.max(np.abs(got / got64 - 1.0)) <= 1e-8


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_df_presweeps_solve_to_planted_x(solver):
    n = 1500
    P = W.dense_householder(4 * n, n, n - 100, 1e6, 1e-4, seed=3)
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), solver=solver, seed=4, svd_mode=L.LSRN_SVD_DF)
    assert info["rank"] == n - 100
    assert info["jacobi_sweeps_df"] >= 3
    # quadratic convergence from the double-float result: few FP64 sweeps
    assert 1 <= info["jacobi_sweeps"] <= 4
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10


def test_df_presweeps_fat_and_zero_rows():
    # m < n (Algorithm 2) with exactly zero columns of A^T: R has zero rows,
    # which the sweeps must leave alone
    m, n = 1300, 5200
    rng = np.random.default_rng(17)
    A = rng.standard_normal((m, n))
    A[::7] = 0.0
    b = rng.standard_normal(m)
    x, info = L.solve(_dev(A), _dev(b), seed=8, svd_mode=L.LSRN_SVD_DF)
    keep = np.any(A != 0.0, axis=1)
    assert info["rank"] == int(keep.sum())
    assert info["jacobi_sweeps_df"] >= 1
    xs = O.minlen_svd(A, b)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10


def test_df_presweeps_only_in_their_range():
    P = W.dense_householder(3000, 1000, 1000, 1e3, 1e-4, seed=2)   # q = 1000: FP64 sweeps only
    _, info = L.solve(_dev(P.A), _dev(P.b), seed=1, svd_mode=L.LSRN_SVD_DF)
    assert info["jacobi_sweeps_df"] == 0 and info["jacobi_sweeps"] > 0
    P2 = W.dense_householder(4000, 1100, 1100, 1e3, 1e-4, seed=2)   # q = 1100, FP64 by default
    _, info = L.solve(_dev(P2.A), _dev(P2.b), seed=1)
    assert info["jacobi_sweeps_df"] == 0
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_plan(_dev(P.A), L.default_options(svd_mode=7))
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
