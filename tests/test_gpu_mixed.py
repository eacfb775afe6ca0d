"""Mixed-precision iteration (LSRN_ITER_F32): passes over an FP32 copy of A,
double-double refinement against the FP64 A.  The result must meet the same
accuracy as the FP64 path against the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
@pytest.mark.parametrize("sketch", [0, 1])
def test_mixed_c1(solver, sketch):
    P = W.c1_problem(0)
    xs, _ = O.minlen_refined(P.A, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), solver=solver, seed=0, sketch_mode=sketch,
                      iter_mode=L.LSRN_ITER_F32)
    x = x.cpu().numpy()
    assert info["rank"] == 80
    assert 1 <= info["refine_steps"] <= 6
    assert O.rel_err(x, xs) <= 1e-10
    r = O.dd_residual(P.A, P.b, x)
    assert np.linalg.norm(O.dd_atr(P.A, r)) / np.linalg.norm(r) <= 1e-12


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_mixed_fat_and_ridge(solver):
    # m < n keeps FP64 passes (the option is ignored there); m >= n ridge uses FP32 passes
    P = W.dense_haar(1500, 70, 55, 1e5, 0.0, seed=4)
    A = np.ascontiguousarray(P.A.T)
    b = A @ np.random.Generator(np.random.PCG64(5)).standard_normal(1500)
    xs, _ = O.minlen_refined(A, b)
    x, info = L.solve(_dev(A), _dev(b), solver=solver, seed=1, iter_mode=L.LSRN_ITER_F32)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10
    rng = np.random.Generator(np.random.PCG64(6))
    for shape in [(900, 40), (40, 900)]:
        A = rng.standard_normal(shape)
        b = rng.standard_normal(shape[0])
        x, _ = L.solve(_dev(A), _dev(b), solver=solver, lambda_=1e-2, seed=2,
                       iter_mode=L.LSRN_ITER_F32)
        assert O.rel_err(x.cpu().numpy(), O.ridge_closed_form(A, b, 1e-2)) <= 1e-10


def test_mixed_householder_medium():
    P = W.dense_householder(40_000, 300, 270, 1e6, 1e-4, seed=2)
    xf = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), seed=1, sketch_mode=L.LSRN_SKETCH_TC_SLICED,
                      iter_mode=L.LSRN_ITER_F32)
    assert O.rel_err(x.cpu().numpy(), xf) <= 1e-10
