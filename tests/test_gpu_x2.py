"""Double-float iteration (LSRN_ITER_F32X2): A kept as two FP32 planes
(hi + lo = A / 2^e to 48 bits), every pass on the FP32 pipe with error-free
products and sums, refinement in double-double on the FP64 A.  Results must
meet the FP64 path's accuracy against the oracle: relative error <= 1e-10 and
normal-equation residual <= 1e-12, for m >= n and m < n, LSQR and CS."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")

def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _ne_resid(A, b, x):
    r = O.dd_residual(A, b, x)
    rn = np.linalg.norm(r)
    if rn == 0.0:
        return 0.0
    return np.linalg.norm(O.dd_atr(A, r)) / (O.two_norm_estimate(A) * rn)


def _solve(A, b, **kw):
    x, info = L.solve(_dev(A), _dev(b), iter_mode=L.LSRN_ITER_F32X2, **kw)
    return x.cpu().numpy(), info


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
@pytest.mark.parametrize("m,n", [(20_000, 600), (12_001, 1031), (9000, 2000)])
def test_x2_tall_householder(solver, m, n):
    P = W.dense_householder(m, n, n - 40, 1e6, 1e-4, seed=m % 97)
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    x, info = _solve(P.A, P.b, solver=solver, seed=3)
    assert info["rank"] == n - 40
    assert O.rel_err(x, xs) <= 1e-10
    assert _ne_resid(P.A, P.b, x) <= 1e-12


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_x2_short_sweep_then_refinement(solver):
    # the double-float sweep stops at 1e-8 and two refinement steps finish the
    # job: fewer sweep iterations than FP64 mode, the same accuracy
    P = W.dense_householder(15_000, 700, 650, 1e6, 1e-4, seed=8)
    _, i64 = L.solve(_dev(P.A), _dev(P.b), solver=solver, seed=1)
    x, i2 = _solve(P.A, P.b, solver=solver, seed=1)
    assert i2["iterations"] < i64["iterations"]
    assert i2["refine_steps"] == 2
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    assert O.rel_err(x, xs) <= 1e-10
    assert _ne_resid(P.A, P.b, x) <= 1e-12


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_x2_fat(solver):
    # m < n: x is iterated in R^n; 2^-48 rounding of A keeps null(A) out to ~1e-15
    P = W.dense_householder(30_000, 700, 660, 1e5, 0.0, seed=11)
    A = np.ascontiguousarray(P.A.T)                 # 700 x 30000 = V Sigma U^T
    b = np.random.Generator(np.random.PCG64(12)).standard_normal(700)
    xs = O.minlen_from_factors(P.apply_Vt, P.sigma, P.apply_U, b)
    x, info = _solve(A, b, solver=solver, seed=2)
    assert info["tall"] == 0 and info["rank"] == 660
    assert O.rel_err(x, xs) <= 1e-10
    assert _ne_resid(A, b, x) <= 1e-12


@pytest.mark.parametrize("shape", [(8000, 600), (600, 8000)])
def test_x2_ridge(shape):
    rng = np.random.Generator(np.random.PCG64(21))
    A = rng.standard_normal(shape)
    b = rng.standard_normal(shape[0])
    for solver in ("lsqr", "cs"):
        x, _ = _solve(A, b, solver=solver, lambda_=1e-2, seed=5)
        assert O.rel_err(x, O.ridge_closed_form(A, b, 1e-2)) <= 1e-10


@pytest.mark.parametrize("scale", [2.0 ** -300, 1e-60, 3e80])
def test_x2_extreme_scales(scale):
    # the planes hold A / 2^e: matrices far outside the FP32 range solve as well
    # (scales whose squares stay inside the FP64 range, which the SVD needs)
    P = W.dense_householder(6000, 600, 600, 1e4, 1e-3, seed=31)
    A = P.A * scale
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b) / scale
    x, info = _solve(A, P.b, seed=4)
    assert np.all(np.isfinite(x))
    assert O.rel_err(x, xs) <= 1e-10


@pytest.mark.parametrize("n", [512, 513, 4096])
def test_x2_short_side_limits(n):
    # q <= 512 runs FP64 passes, q in (512, 4096] the double-float pass
    P = W.dense_householder(3 * n + 7, n, n, 1e5, 1e-4, seed=n)
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    x, _ = _solve(P.A, P.b, seed=6)
    assert O.rel_err(x, xs) <= 1e-10


def test_dense_short_side_above_4096_is_unsupported():
    A = torch.zeros((4200, 4097), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_plan(A, L.default_options(iter_mode=L.LSRN_ITER_F32X2))
    assert e.value.status == L.LSRN_ERR_UNSUPPORTED


def test_x2_zero_matrix():
    A = np.zeros((3000, 700))
    b = np.ones(3000)
    x, info = _solve(A, b)
    assert info["rank"] == 0 and not np.any(x)


def test_x2_tc_sketch_plan_reuse():
    P = W.dense_householder(20_000, 800, 760, 1e6, 1e-4, seed=41)
    plan = L.lsrn_plan(_dev(P.A), L.default_options(seed=9, sketch_mode=L.LSRN_SKETCH_TC_SLICED,
                                                     iter_mode=L.LSRN_ITER_F32X2))
    try:
        rng = np.random.Generator(np.random.PCG64(42))
        for k in range(3):
            b = P.b if k == 0 else rng.standard_normal(20_000)
            x, _ = L.lsrn_solve_lsqr(plan, _dev(b))
            xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, b)
            assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10
    finally:
        plan.close()
