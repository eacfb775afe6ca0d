"""Pins for the oracle's min-length solution x* (section 1, eq. ls_min_length;
section 2.1) and its SVD, against facts fixed independently of the oracle:
the four Penrose conditions, closed-form pseudoinverses, an independent
factorisation (complete orthogonal decomposition), LAPACK's SVD and lstsq, the
generator's planted factors, exact rational arithmetic, and the optimality
conditions A^T(b - Ax) = 0, x in range(A^T)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as W


def _planted(m, n, r, seed, integer=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    if integer:
        L = rng.integers(-3, 4, size=(m, r)).astype(float)
        R = rng.integers(-3, 4, size=(r, n)).astype(float)
    else:
        L = rng.standard_normal((m, r))
        R = rng.standard_normal((r, n))
    return L @ R


@pytest.mark.parametrize("shape,r,seed", [((8, 5), 3, 0), ((5, 8), 2, 1), ((7, 7), 4, 2),
                                          ((6, 3), 3, 3), ((3, 6), 1, 4)])
def test_penrose_conditions(shape, r, seed):
    A = _planted(*shape, r, seed, integer=True)
    X = O.pinv_svd(A, rcond=1e-10)
    tol = 1e-11 * max(1.0, np.abs(A).max()) ** 2
    assert np.allclose(A @ X @ A, A, atol=tol)
    assert np.allclose(X @ A @ X, X, atol=tol)
    assert np.allclose((A @ X).T, A @ X, atol=tol)
    assert np.allclose((X @ A).T, X @ A, atol=tol)


def test_rank_one_closed_form():
    rng = np.random.Generator(np.random.PCG64(3))
    u, v = rng.standard_normal(9), rng.standard_normal(4)
    A = np.outer(u, v)
    X = O.pinv_svd(A, rcond=1e-12)
    ref = np.outer(v, u) / (u @ u) / (v @ v)
    assert np.allclose(X, ref, rtol=1e-12, atol=1e-14)


def test_orthonormal_columns_and_diagonal():
    rng = np.random.Generator(np.random.PCG64(4))
    Q, _ = np.linalg.qr(rng.standard_normal((12, 5)))
    assert np.allclose(O.pinv_svd(Q), Q.T, atol=1e-14)
    D = np.diag([3.0, 0.0, -2.0, 0.5])
    ref = np.diag([1 / 3.0, 0.0, -0.5, 2.0])
    assert np.allclose(O.pinv_svd(D), ref, atol=1e-15)
    b = np.array([1.0, 2.0, 3.0, 4.0])
    assert np.allclose(O.minlen_svd(D, b), ref @ b, atol=1e-15)


def test_jacobi_svd_against_lapack():
    rng = np.random.Generator(np.random.PCG64(8))
    for shape in [(30, 7), (7, 30), (20, 20)]:
        A = rng.standard_normal(shape) @ np.diag(np.logspace(0, -8, shape[1]))
        U, s, V = O.jacobi_svd(A)
        ref = np.linalg.svd(A, compute_uv=False)
        k = min(shape)
        assert np.allclose(s[:k], ref[:k], rtol=1e-12, atol=1e-15 * ref[0])
        assert np.allclose(U[:, :k].T @ U[:, :k], np.eye(k), atol=1e-10)
        assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)
        assert np.allclose((U[:, :k] * s[:k]) @ V[:, :k].T, A, atol=1e-13)


def test_minlen_independent_routes_agree():
    # SVD route vs complete orthogonal factorisation vs LAPACK gelsd (section 2.1)
    for (m, n, r, seed) in [(60, 12, 9, 0), (12, 60, 9, 1), (40, 40, 25, 2)]:
        A = _planted(m, n, r, seed)
        b = np.random.Generator(np.random.PCG64(seed + 50)).standard_normal(m)
        xs = O.minlen_svd(A, b, rcond=1e-10)
        xc = O.minlen_cod(A, b, rcond=1e-10)
        xl = np.linalg.lstsq(A, b, rcond=1e-10)[0]
        assert O.rel_err(xc, xs) < 1e-12
        assert O.rel_err(xl, xs) < 1e-12


def test_minlen_optimality_conditions():
    A = _planted(50, 10, 6, 11)
    b = np.random.Generator(np.random.PCG64(12)).standard_normal(50)
    x = O.minlen_svd(A, b, rcond=1e-10)
    r = b - A @ x
    assert np.linalg.norm(A.T @ r) < 1e-12 * np.linalg.norm(A) * np.linalg.norm(r)
    # x in range(A^T): orthogonal to an explicit null-space basis
    _, s, Vt = np.linalg.svd(A)
    null = Vt[6:].T
    assert np.linalg.norm(null.T @ x) < 1e-12 * np.linalg.norm(x)
    # minimal norm: adding a null-space vector makes x longer, keeps the residual
    z = x + null @ np.ones(null.shape[1])
    assert np.linalg.norm(b - A @ z) == pytest.approx(np.linalg.norm(r), rel=1e-10)
    assert np.linalg.norm(z) > np.linalg.norm(x)


def test_dd_residual_exact_on_integers():
    rng = np.random.Generator(np.random.PCG64(13))
    A = rng.integers(-2 ** 26, 2 ** 26, size=(6, 5)).astype(float)
    x = rng.integers(-2 ** 26, 2 ** 26, size=5).astype(float) * 2.0 ** -20
    b = rng.integers(-2 ** 26, 2 ** 26, size=6).astype(float)
    r = O.dd_residual(A, b, x)
    g = O.dd_atr(A, r)
    for i in range(6):
        exact = Fraction(b[i]) - sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(5))
        assert r[i] == float(exact)
    for j in range(5):
        exact = sum(Fraction(A[i, j]) * Fraction(r[i]) for i in range(6))
        assert g[j] == float(exact)


def test_refined_minlen_on_planted_problem():
    # The 2000 x 100 rank-80 recipe (cond 1e6, noise 1e-3): the refined x*
    # satisfies the normal equations to double-double accuracy, agrees with the
    # independent COD route and the planted factors to the FP64 floor, and lies
    # in range(A^T) = range(V).
    P = W.c1_problem(0)
    A, b = P.A, P.b
    x, corr = O.minlen_refined(A, b, steps=3)
    assert corr[-1] < 1e-12 * np.linalg.norm(x)
    r = O.dd_residual(A, b, x)
    g = O.dd_atr(A, r)
    assert np.linalg.norm(g) / (np.linalg.norm(r)) < 1e-12         # ||A||_2 = 1 here
    assert O.rel_err(O.minlen_cod(A, b), x) < 3e-10
    assert O.rel_err(O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, b), x) < 3e-10
    V = P.meta["V"]
    assert np.linalg.norm(x - V @ (V.T @ x)) < 1e-10 * np.linalg.norm(x)


def test_generator_spectrum():
    P = W.dense_householder(3000, 40, 30, 1e6, 1e-4, seed=5)
    s = np.linalg.svd(P.A, compute_uv=False)
    assert np.allclose(s[:30], P.sigma, rtol=1e-9)
    assert s[30] < 1e-14
    V = P.meta["V"]
    assert np.allclose(V.T @ V, np.eye(30), atol=1e-13)


def test_ridge_closed_form_is_augmented_minlen():
    # Section 5: min ||Ax-b||^2 + ||lam x||^2 == LS on [A; lam I] == x = z/lam of
    # the min-length solution of [A/lam, I] [z; r] = b.
    rng = np.random.Generator(np.random.PCG64(21))
    for (m, n) in [(40, 9), (9, 40)]:
        A = rng.standard_normal((m, n))
        b = rng.standard_normal(m)
        lam = 0.3
        x = O.ridge_closed_form(A, b, lam)
        x_tall = O.minlen_svd(np.vstack([A, lam * np.eye(n)]), np.concatenate([b, np.zeros(n)]))
        zr = O.minlen_svd(np.hstack([A / lam, np.eye(m)]), b)
        assert O.rel_err(x_tall, x) < 1e-12
        assert O.rel_err(zr[:n] / lam, x) < 1e-12
