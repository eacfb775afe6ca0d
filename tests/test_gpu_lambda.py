"""Sketch reuse across the Tikhonov lambda (section 5): a plan created with
lambda > 0 keeps the unaugmented part of its sketch, and lsrn_plan_set_lambda
rebuilds A~ for a new lambda from it (G_1 A + lambda G_2 for m >= n,
A G_1 / lambda + G_2 for m < n).  The rebuilt sketch must equal a fresh plan's
sketch at the sketch tolerance, and each solve the ridge closed form
(A^T A + lambda^2 I)^-1 A^T b."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _sketch(A, lam, seed, mode):
    plan = L.lsrn_plan(A, L.default_options(seed=seed, lambda_=lam, sketch_mode=mode))
    L.lsrn_sketch(plan)
    S = L.lsrn_plan_get_sketch(plan)
    plan.close()
    return S


@pytest.mark.parametrize("shape,solver,mode", [((3000, 120), "lsqr", "tc"), ((3000, 120), "cs", "f64"),
                                               ((90, 1600), "lsqr", "f64"), ((90, 1600), "cs", "tc")])
def test_lambda_sweep_reuses_the_sketch(shape, solver, mode):
    m, n = shape
    q = min(m, n)
    P = W.dense_householder(max(m, n), q, rank=q, cond=1e4, noise=1e-2, seed=141)
    A_h = P.A if m >= n else np.ascontiguousarray(P.A.T)
    b_h = P.b if m >= n else np.random.Generator(np.random.PCG64(142)).standard_normal(m)
    A, b = torch.from_numpy(A_h).cuda(), torch.from_numpy(b_h).cuda()
    smode = L.LSRN_SKETCH_TC_SLICED if mode == "tc" else L.LSRN_SKETCH_F64
    fn = L.lsrn_solve_lsqr if solver == "lsqr" else L.lsrn_solve_cs
    plan = L.lsrn_plan(A, L.default_options(seed=3, lambda_=0.3, sketch_mode=smode))
    try:
        for k, lam in enumerate([0.3, 1e-2, 1.5, 1e-3]):
            if k:
                L.lsrn_plan_set_lambda(plan, lam)
                S = L.lsrn_plan_get_sketch(plan)
                S2 = _sketch(A, lam, 3, smode)
                assert np.linalg.norm(S - S2) <= 1e-13 * np.linalg.norm(S2)
            x, info = fn(plan, b)
            ref = O.ridge_closed_form(A_h, b_h, lam)
            assert O.rel_err(x.cpu().numpy(), ref) <= 1e-10, (lam, info)
    finally:
        plan.close()


def test_set_lambda_rejects_plans_without_ridge():
    A = torch.randn(500, 20, dtype=torch.float64, device="cuda")
    plan = L.lsrn_plan(A, L.default_options(seed=1))
    try:
        with pytest.raises(L.LsrnError) as e:
            L.lsrn_plan_set_lambda(plan, 0.1)
        assert e.value.status == L.LSRN_ERR_INVALID_ARG
    finally:
        plan.close()
    plan = L.lsrn_plan(A, L.default_options(seed=1, lambda_=0.5))
    try:
        for bad in (0.0, -1.0, float("inf")):
            with pytest.raises(L.LsrnError):
                L.lsrn_plan_set_lambda(plan, bad)
    finally:
        plan.close()
