"""GPU parity of the tensor-core sketch (exact bf16 digit slices on tcgen05,
FP64 accumulation of exact chunk sums) against the oracle's FP64 sketch and
through full solves."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _oracle_sketch(A, seed, lam=0.0):
    m, n = A.shape
    if m >= n:
        B = np.vstack([A, lam * np.eye(n)]) if lam > 0 else A
        return O.sketch_block(seed, 0, 0, B.shape[0], math.ceil(2 * n)).T @ B
    B = np.hstack([A / lam, np.eye(m)]) if lam > 0 else A
    return (B @ O.sketch_block(seed, 0, 0, B.shape[1], math.ceil(2 * m))).T


def _tc_sketch(A, seed, lam=0.0):
    plan = L.lsrn_plan(_dev(A), L.default_options(seed=seed, lambda_=lam,
                                                  sketch_mode=L.LSRN_SKETCH_TC_SLICED))
    L.lsrn_sketch(plan)
    S = L.lsrn_plan_get_sketch(plan)
    plan.close()
    return S


@pytest.mark.parametrize("m,n,lam", [(128, 64, 0.0), (2000, 100, 0.0), (777, 37, 0.0),
                                     (3000, 200, 0.0), (1100, 513, 0.0), (40, 900, 0.0),
                                     (501, 64, 0.3), (40, 450, 0.2)])
def test_tc_sketch_matches_oracle(m, n, lam):
    rng = np.random.Generator(np.random.PCG64(m + 3 * n))
    A = rng.standard_normal((m, n))
    S = _tc_sketch(A, 5, lam)
    ref = _oracle_sketch(A, 5, lam)
    assert np.linalg.norm(S - ref) <= 1e-13 * np.linalg.norm(ref)


def test_tc_sketch_many_segments(monkeypatch):
    monkeypatch.setenv("LSRN_TC_SEGMENT_ROWS", "192")
    rng = np.random.Generator(np.random.PCG64(2))
    A = rng.standard_normal((1500, 96))
    S = _tc_sketch(A, 9)
    ref = _oracle_sketch(A, 9)
    assert np.linalg.norm(S - ref) <= 1e-13 * np.linalg.norm(ref)


def test_tc_sketch_columns_of_wildly_different_scale():
    # per-column exponents: each column of the sketch keeps FP64 relative accuracy
    rng = np.random.Generator(np.random.PCG64(3))
    A = rng.standard_normal((900, 40)) * np.logspace(-150, 150, 40)
    A[:, 7] = 0.0
    S = _tc_sketch(A, 1)
    ref = _oracle_sketch(A, 1)
    for j in range(40):
        nr = np.linalg.norm(ref[:, j])
        if nr == 0:
            assert np.all(S[:, j] == 0)
        else:
            assert np.linalg.norm(S[:, j] - ref[:, j]) <= 1e-13 * nr


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_tc_solve_c1(solver):
    P = W.c1_problem(0)
    xs, _ = O.minlen_refined(P.A, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), solver=solver, seed=0,
                      sketch_mode=L.LSRN_SKETCH_TC_SLICED)
    assert info["rank"] == 80
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10


def test_tc_solve_householder_medium():
    P = W.dense_householder(40_000, 300, 270, 1e6, 1e-4, seed=2)
    xf = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), seed=1, sketch_mode=L.LSRN_SKETCH_TC_SLICED)
    assert info["rank"] == 270
    assert O.rel_err(x.cpu().numpy(), xf) <= 1e-10


def test_tc_sketch_column_maxima_just_below_a_power_of_two():
    # |X_lj| / 2^e_j close to 1 puts the fixed-point digit split at the edge of
    # its 64-bit range (the first digit rounds to 128)
    rng = np.random.Generator(np.random.PCG64(17))
    A = rng.standard_normal((1500, 120))
    for j in range(120):
        k = 1 + j % 53
        A[rng.integers(0, 1500), j] = (1.0 - 2.0 ** -k) * 2.0 ** (j % 7 - 3) * (-1) ** j
    S = _tc_sketch(A, 4)
    ref = _oracle_sketch(A, 4)
    for j in range(120):
        assert np.linalg.norm(S[:, j] - ref[:, j]) <= 1e-13 * np.linalg.norm(ref[:, j])
