"""Pins for the oracle's ||A||_2 estimate (``two_norm_estimate``), the
denominator of the normal-equation criterion ||A^T r|| / (||A||_2 ||r||) that
every solve is judged by.

What fixes the value independently of the oracle:
  * the planted largest singular value of A = U diag(sigma) V^T (closed form);
  * LAPACK's SVD (numpy.linalg.norm(A, 2)) and the oracle's own one-sided
    Jacobi SVD (itself pinned against LAPACK);
  * the Rayleigh bound: for a unit v, ||A^T A v||^(1/2) <= sigma_1, so power
    iteration never overestimates sigma_1.

Cases: dense tall, dense fat, and scipy-sparse storage.  Planted slips (the
Frobenius norm, the squared norm, a single iteration) must each fail one of the
pins, so the pins would catch them in the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O


def _planted(m, n, sigma, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    k = len(sigma)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return (U * np.asarray(sigma)) @ V.T


def _gap_spectrum(k, top=3.0):
    # sigma_1 = 3, then a gap of 2x and a log-spaced tail: 30 power iterations
    # reduce the error of sigma_1^2 by (1/2)^60
    return np.concatenate([[top], 0.5 * top * np.logspace(0, -4, k - 1)])


def _cases():
    out = []
    out.append(("dense tall", _planted(400, 30, _gap_spectrum(30), 1), 3.0))
    out.append(("dense fat", _planted(25, 500, _gap_spectrum(25, 7.5), 2), 7.5))
    S = sp.random(3000, 200, density=0.01, format="csr",
                  random_state=np.random.RandomState(5), data_rvs=np.random.RandomState(6).randn)
    s2 = np.linalg.norm(S.toarray(), 2)
    spike = sp.csr_matrix(([4.0 * s2], ([7], [11])), shape=S.shape)   # sigma_1 ~ 4 s2, gap >= 3x
    out.append(("scipy sparse", (S + spike).tocsr(), None))
    return out


def _pins_hold(est_fn) -> bool:
    """All pins for one estimator: within 1e-8 of the planted sigma_1, of
    LAPACK's and of the oracle Jacobi's sigma_1, and never above sigma_1."""
    for _, A, planted in _cases():
        dense = A.toarray() if sp.issparse(A) else A
        lapack = float(np.linalg.norm(dense, 2))
        jac = float(O.jacobi_svd(np.ascontiguousarray(dense if dense.shape[0] >= dense.shape[1]
                                                      else dense.T))[1][0])
        est = float(est_fn(A))
        refs = [lapack, jac] + ([planted] if planted is not None else [])
        if any(abs(est - r) > 1e-8 * r for r in refs):
            return False
        if est > lapack * (1 + 1e-13):
            return False
    return True


def test_two_norm_estimate_matches_planted_lapack_and_jacobi():
    assert _pins_hold(O.two_norm_estimate)


@pytest.mark.parametrize("m,n,seed", [(300, 40, 0), (40, 300, 1), (120, 120, 2)])
def test_two_norm_estimate_never_exceeds_sigma1(m, n, seed):
    # random Gaussian matrices have a small gap between sigma_1 and sigma_2, so
    # the estimate may be short of sigma_1, but never above it
    A = np.random.Generator(np.random.PCG64(seed)).standard_normal((m, n))
    s1 = float(np.linalg.norm(A, 2))
    est = O.two_norm_estimate(A)
    assert est <= s1 * (1 + 1e-13)
    assert est >= 0.9 * s1


@pytest.mark.parametrize("slip", [
    lambda A: float(sp.linalg.norm(A) if sp.issparse(A) else np.linalg.norm(A, "fro")),
    lambda A: O.two_norm_estimate(A) ** 2,
    lambda A: O.two_norm_estimate(A, iters=1),
], ids=["frobenius", "squared", "one_iteration"])
def test_planted_slips_fail_the_pins(slip):
    assert not _pins_hold(slip)
