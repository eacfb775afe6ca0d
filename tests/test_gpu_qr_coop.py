"""Householder QR of the sketch in one cooperative launch (short sides up to
3000).  After lsrn_precond the plan's sketch buffer holds R in its upper
triangle; R must be LAPACK's R of the same sketch (numpy.linalg.qr, a library
routine) up to rounding, with rows of near-zero diagonal allowed a sign flip
(the same reflector convention, beta = -sign(alpha) ||x||, fixes the sign of
every well-defined row)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("m,n,rank", [(6000, 700, 650), (9000, 1031, 1031), (3001, 37, 30),
                                      (12000, 2000, 1800)])
def test_cooperative_qr_matches_lapack(m, n, rank):
    P = W.dense_householder(m, n, rank, 1e6, 1e-4, seed=n % 83)
    plan = L.lsrn_plan(_dev(P.A), L.default_options(seed=3))
    try:
        L.lsrn_sketch(plan)
        S = L.lsrn_plan_get_sketch(plan)
        r = L.lsrn_precond(plan)
        X = L.lsrn_plan_get_sketch(plan)      # now the factored sketch
    finally:
        plan.close()
    assert r == rank
    q = S.shape[1]
    Rg = np.triu(X[:q])
    Rn = np.linalg.qr(S, mode="r")
    # row signs from the diagonal (only rows of negligible diagonal can differ)
    sg = np.sign(np.diag(Rg)) * np.sign(np.diag(Rn))
    sg[sg == 0] = 1.0
    scale = np.linalg.norm(Rn)
    assert np.linalg.norm(Rg * sg[:, None] - Rn) <= 1e-12 * scale
    big = np.abs(np.diag(Rn)) > 1e-8 * np.abs(np.diag(Rn)).max()
    assert np.all(sg[big] == 1.0)
