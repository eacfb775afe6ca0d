"""QR preconditioner for full-rank (ridge) problems: N = R^-1 from the sketch's
QR factorisation (LSRN_PRECOND_QR).  With A~ = QR and R = U_R Sigma V^T,
A R^-1 = (A V Sigma^-1) U_R^T, so the preconditioned matrix has exactly the
singular values of the SVD preconditioner's (Lemma 4.3) and the same CS bounds.
Checked: R^-1 R = I for block counts with ragged tails; sigma(B N_qr) =
sigma(B N_svd) for the same G; ridge solves match the closed form; the mode is
refused without lambda."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _augmented(A, lam):
    m, n = A.shape
    return np.vstack([A, lam * np.eye(n)]) if m >= n else np.hstack([A / lam, np.eye(m)])


@pytest.mark.parametrize("m,n", [(2000, 130), (5000, 700), (90, 1600)])
def test_r_inverse_and_preconditioned_spectrum(m, n):
    rng = np.random.Generator(np.random.PCG64(m + n))
    A = rng.standard_normal((m, n)) * np.logspace(0, -3, n)[None, :]
    lam = 0.05
    At = torch.from_numpy(A).cuda()
    plans = {}
    for mode in (L.LSRN_PRECOND_QR, L.LSRN_PRECOND_SVD):
        plan = L.lsrn_plan(At, L.default_options(seed=9, lambda_=lam, precond_mode=mode))
        L.lsrn_sketch(plan)
        L.lsrn_precond(plan)
        N, sig = L.lsrn_plan_get_precond(plan)
        R = np.triu(L.lsrn_plan_get_sketch(plan)[: N.shape[0]])     # factored in place
        plans[mode] = (N, sig, R)
        plan.close()
    Nq, dq, R = plans[L.LSRN_PRECOND_QR]
    q = Nq.shape[0]
    assert Nq.shape == (q, q)
    assert np.linalg.norm(Nq @ R - np.eye(q)) <= 1e-12 * np.linalg.cond(R)
    assert np.allclose(np.sort(dq)[::-1], np.sort(np.abs(np.diag(R)))[::-1], rtol=0, atol=0)
    B = _augmented(A, lam)
    Ns = plans[L.LSRN_PRECOND_SVD][0]
    if m >= n:
        s_qr, s_svd = np.linalg.svd(B @ Nq, compute_uv=False), np.linalg.svd(B @ Ns, compute_uv=False)
    else:
        s_qr, s_svd = np.linalg.svd(Nq.T @ B, compute_uv=False), np.linalg.svd(Ns.T @ B, compute_uv=False)
    assert np.allclose(s_qr, s_svd, rtol=1e-10, atol=0)


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
@pytest.mark.parametrize("shape", [(3000, 120), (150, 2500)])
def test_ridge_solves_with_r_inverse(solver, shape):
    m, n = shape
    q = min(m, n)
    P = W.dense_householder(max(m, n), q, rank=q, cond=1e5, noise=1e-2, seed=151)
    A = P.A if m >= n else np.ascontiguousarray(P.A.T)
    b = P.b if m >= n else np.random.Generator(np.random.PCG64(152)).standard_normal(m)
    for lam in (1e-3, 0.3):
        x, info = L.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), solver=solver,
                          seed=5, lambda_=lam, precond_mode=L.LSRN_PRECOND_QR)
        assert info["rank"] == q and info["jacobi_sweeps"] == 0
        assert O.rel_err(x.cpu().numpy(), O.ridge_closed_form(A, b, lam)) <= 1e-10


def test_qr_mode_needs_lambda():
    A = torch.randn(400, 30, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_plan(A, L.default_options(precond_mode=L.LSRN_PRECOND_QR))
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
