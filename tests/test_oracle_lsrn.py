"""Pins for the oracle's LSRN (Algorithms 1-3, Theorems 4.2-4.6, section 5).

Each check compares the oracle with something it does not compute itself: the
Chebyshev polynomial in closed form, iteration counts printed in the paper
(tests/golden), scipy's independent LSQR, CG on the normal equations, the
singular values of G U for the exact G (Lemma 4.3), the probability statement
of Theorem 4.5, and the ridge closed form."""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cheb_T(k, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    big = np.abs(x) > 1
    out[~big] = np.cos(k * np.arccos(x[~big]))
    out[big] = np.cosh(k * np.arccosh(np.abs(x[big]))) * np.where(x[big] < 0, (-1) ** k, 1)
    return out


@pytest.mark.parametrize("tol", [1e-1, 1e-3, 1e-6, 1e-10])
def test_chebyshev_matches_polynomial_closed_form(tol):
    # For B = diag(d) the CS residual after j steps is P_j(d^2) * b with
    # P_j(l) = T_j((dbar - l)/cbar) / T_j(dbar/cbar)  (Alg. 3 is Chebyshev
    # acceleration on the normal equations with spectrum [sL^2, sU^2]).
    rng = np.random.Generator(np.random.PCG64(1))
    d = np.sort(rng.uniform(0.5, 2.0, 40))
    d[0], d[-1] = 0.5, 2.0
    b = rng.standard_normal(40)
    x, info = O.chebyshev(lambda v: d * v, lambda v: d * v, b, 40, 0.5, 2.0, tol)
    j = info["iterations"]
    dbar, cbar = info["d"], info["c"]
    ref = _cheb_T(j, (dbar - d * d) / cbar) / _cheb_T(j, np.array([dbar / cbar]))[0] * b
    r = b - d * x
    assert np.max(np.abs(r - ref)) < 1e-13 * max(1.0, np.max(np.abs(b)))


def test_literal_alpha1_breaks_the_closed_form(monkeypatch):
    # Planted mistake: Algorithm 3 as printed (alpha = d - c^2/(2d) at k = 1)
    # no longer reproduces the Chebyshev polynomial -- the pin above catches it.
    def cheb_literal(matvec, rmatvec, b, n, sL, sU, tol):
        d = 0.5 * (sU * sU + sL * sL)
        c = 0.5 * (sU * sU - sL * sL)
        K = O.cs_iteration_count(sL, sU, tol)
        x = np.zeros(n); v = np.zeros(n); r = b.copy(); a = 0.0
        for k in range(K + 1):
            if k == 0:
                be, a = 0.0, 1.0 / d
            elif k == 1:
                be, a = 0.5 * (c / d) ** 2, d - c * c / (2.0 * d)
            else:
                be = (a * c / 2.0) ** 2
                a = 1.0 / (d - a * c * c / 4.0)
            v = be * v + rmatvec(r); x = x + a * v; r = r - a * matvec(v)
        return x, dict(iterations=K + 1, d=d, c=c)
    monkeypatch.setattr(O, "chebyshev", cheb_literal)
    with pytest.raises(AssertionError):
        test_chebyshev_matches_polynomial_closed_form(1e-6)


def _golden_table3():
    rows = []
    with open(os.path.join(GOLDEN, "table3_iterations.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, m3, m2, r2, cs, lsqr = line.split()
                rows.append((name, int(m3), None if m2 == "-" else int(m2),
                             None if r2 == "-" else int(r2), int(cs), int(lsqr)))
    return rows


def test_table3_chebyshev_count():
    # gamma = 2, eps = 1e-14, bounds of Theorem 4.5 with alpha = 1/sqrt(s):
    # the loop k = 0..K runs K + 1 = 106 times (Table 3).
    for name, m3, m2, r2, cs_iters, lsqr_iters in _golden_table3():
        cases = [(m3, m3)] + ([(m2, r2)] if m2 else [])
        for m, r in cases:
            s = math.ceil(2.0 * m)
            sL, sU = O.thm45_bounds(r, s, 1.0 / math.sqrt(s))
            assert O.cs_iteration_count(sL, sU, 1e-14) + 1 == cs_iters, (name, m, r)
            # LSQR's printed count lies below Theorem 4.6's bound
            assert lsqr_iters <= O.thm46_bound(r, s, 1e-14)


def test_section_numbers():
    vals = {}
    with open(os.path.join(GOLDEN, "section_numbers.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                vals[k] = float(v)
    assert O.thm45_kappa_bound(1, 2, 0.0) < vals["kappa_bound_at_half_upper"]
    assert O.thm45_kappa_bound(1000, 2001, 0.0) < vals["kappa_bound_at_half_upper"]
    it = O.thm46_bound(1, 2, vals["tolerance"])
    assert abs(it - vals["niter_gamma2_eps1e-14"]) < 0.1 * vals["niter_gamma2_eps1e-14"]


def test_lsqr_matches_scipy_iterates():
    from scipy.sparse.linalg import lsqr as sp_lsqr
    rng = np.random.Generator(np.random.PCG64(2))
    # well-conditioned, so the iterates themselves are well determined in FP64
    A = rng.standard_normal((60, 15)) @ np.diag(np.logspace(0, -1, 15))
    b = rng.standard_normal(60)
    # (iterates just before the Krylov space fills up are sensitive to rounding
    # in any implementation, so compare early iterates and the converged one)
    for k in (1, 2, 5, 8, 10, 30):
        x, _ = O.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 15, atol=0, btol=0, iter_lim=k)
        xs = sp_lsqr(A, b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
        assert O.rel_err(x, xs) < 1e-10, k


def test_lsqr_equals_cg_on_normal_equations():
    rng = np.random.Generator(np.random.PCG64(3))
    A = rng.standard_normal((40, 8))
    b = rng.standard_normal(40)
    K = A.T @ A
    f = A.T @ b
    z = np.zeros(8); r = f.copy(); p = r.copy(); rr = r @ r
    for k in range(1, 7):
        Kp = K @ p; a = rr / (p @ Kp); z = z + a * p; r = r - a * Kp
        rn = r @ r; p = r + (rn / rr) * p; rr = rn
        x, _ = O.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 8, atol=0, btol=0, iter_lim=k)
        assert O.rel_err(x, z) < 1e-9, k


def test_lsqr_terminates_in_rank_steps():
    rng = np.random.Generator(np.random.PCG64(4))
    A = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 10))
    b = rng.standard_normal(30)
    x, info = O.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 10, atol=0, btol=0, iter_lim=3)
    assert O.rel_err(x, O.minlen_svd(A, b, rcond=1e-10)) < 1e-10


def test_lemma43_spectrum_of_AN():
    # sigma(AN) = 1 / sigma(G U) for the very G used by the sketch.
    P = W.dense_haar(400, 30, 20, 1e3, 0.0, seed=7)
    A = P.A
    x, info = O.lsrn(A, P.b, gamma=2.0, seed=3)
    s, r = info["s"], info["rank"]
    assert r == 20
    G = O.sketch_block(3, 0, 0, 400, s).T
    sig_gu = np.linalg.svd(G @ P.meta["U"], compute_uv=False)
    sig_an = np.linalg.svd(A @ info["N"], compute_uv=False)
    assert np.allclose(np.sort(sig_an), np.sort(1.0 / sig_gu), rtol=1e-9)


def test_thm42_seed_independence_and_accuracy():
    P = W.c1_problem(0)
    xr, _ = O.minlen_refined(P.A, P.b)
    for seed in range(4):
        x, info = O.lsrn(P.A, P.b, seed=seed)
        assert info["rank"] == 80
        assert O.rel_err(x, xr) < 2e-9, seed


def test_thm45_probability():
    # P(kappa(AN) > (1+a+sqrt(r/s))/(1-a-sqrt(r/s))) <= 2 exp(-a^2 s / 2)
    P = W.dense_haar(300, 24, 24, 1e4, 0.0, seed=9)
    s = 48
    a = math.sqrt(2.0 * math.log(4.0) / s)       # failure bound 0.5
    bound = O.thm45_kappa_bound(24, s, a)
    fails, kappas = 0, []
    nseeds = 100
    for seed in range(nseeds):
        _, info = O.lsrn(P.A, P.b, gamma=2.0, seed=seed, max_iter=1)
        sv = np.linalg.svd(P.A @ info["N"], compute_uv=False)
        kappas.append(sv[0] / sv[-1])
        fails += kappas[-1] > bound
    assert fails / nseeds <= 2 * math.exp(-a * a * s / 2)
    # and kappa(AN) does not depend on kappa(A) (section 6.2): typical value
    assert np.median(kappas) < O.thm45_kappa_bound(24, s, 0.0)


@pytest.mark.parametrize("cond", [1e2, 1e5, 1e8])
@pytest.mark.parametrize("r", [40, 80, 100])
def test_fig1_iterations_function_of_r_over_s(cond, r):
    # Section 6.2 / Fig. 1: kappa(AN) ~< (1+sqrt(r/s))/(1-sqrt(r/s)) and the LSQR
    # count stays under (log eps - log 2)/log sqrt(r/s), whatever kappa(A).
    P = W.dense_haar(2000, 100, r, cond, 1e-3, seed=int(cond) % 97 + r)
    x, info = O.lsrn(P.A, P.b, gamma=2.0, seed=1)
    s = info["s"]
    assert info["rank"] == r
    assert info["iterations"] <= O.thm46_bound(r, s, 1e-14)
    sv = np.linalg.svd(P.A @ info["N"], compute_uv=False)
    assert sv[0] / sv[-1] <= 1.3 * O.thm45_kappa_bound(r, s, 0.0)


def test_cs_and_lsqr_agree_with_minlen_tall():
    P = W.c1_problem(0)
    xr, _ = O.minlen_refined(P.A, P.b)
    x_l, info_l = O.lsrn(P.A, P.b, solver="lsqr")
    x_c, info_c = O.lsrn(P.A, P.b, solver="cs")
    assert O.rel_err(x_l, xr) < 2e-9 and O.rel_err(x_c, xr) < 2e-9
    sL, sU = info_c["sigma_L"], info_c["sigma_U"]
    assert info_c["iterations"] == O.cs_iteration_count(sL, sU, 1e-14) + 1


def test_fat_algorithm2():
    P = W.dense_haar(1200, 60, 50, 1e4, 1e-3, seed=3)
    A = np.ascontiguousarray(P.A.T)                # 60 x 1200, rank 50
    b = np.random.Generator(np.random.PCG64(4)).standard_normal(60)
    xr, _ = O.minlen_refined(A, b)
    for solver in ("lsqr", "cs"):
        x, info = O.lsrn(A, b, solver=solver, seed=2)
        assert not info["tall"] and info["rank"] == 50 and info["s"] == 120
        assert O.rel_err(x, xr) < 1e-9, solver


@pytest.mark.parametrize("shape", [(500, 30), (30, 500)])
@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_ridge_by_augmentation(shape, solver):
    rng = np.random.Generator(np.random.PCG64(sum(shape)))
    A = rng.standard_normal(shape)
    b = rng.standard_normal(shape[0])
    lam = 1e-1
    x, _ = O.lsrn(A, b, lam=lam, solver=solver, seed=5)
    assert O.rel_err(x, O.ridge_closed_form(A, b, lam)) < 1e-10


def test_rank_zero_returns_zero():
    A = np.zeros((20, 4))
    x, info = O.lsrn(A, np.ones(20))
    assert info["rank"] == 0 and np.all(x == 0)


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_refinement_reaches_target(solver):
    # One refinement step with double-double residuals brings LSRN below the
    # FP64 floor of the 2000 x 100, cond 1e6 problem: ||x - x*|| <= 1e-10 ||x*||
    # and ||A^T r|| / (||A|| ||r||) <= 1e-12 (||A||_2 = 1 for this recipe).
    P = W.c1_problem(0)
    xr, _ = O.minlen_refined(P.A, P.b)
    x, info = O.lsrn(P.A, P.b, solver=solver, refine=1)
    assert info["refine_steps"] == [23]
    assert O.rel_err(x, xr) < 1e-10
    r = O.dd_residual(P.A, P.b, x)
    assert np.linalg.norm(O.dd_atr(P.A, r)) / np.linalg.norm(r) < 1e-12


def test_refinement_fat_and_ridge():
    rng = np.random.Generator(np.random.PCG64(31))
    A = rng.standard_normal((40, 900))
    b = rng.standard_normal(40)
    for lam in (0.0, 1e-3):
        x, _ = O.lsrn(A, b, lam=lam, refine=1, seed=1)
        ref = O.ridge_closed_form(A, b, lam) if lam else O.minlen_svd(A, b)
        assert O.rel_err(x, ref) < 1e-12
