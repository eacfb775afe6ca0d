"""GPU parity of the dense path (Algorithms 1-3, section 5) against the oracle.

Every test calls the CUDA library through its C ABI (python binding) and
compares with the oracle on the same seeded inputs:
  * the sketching matrix bit for bit;
  * the sketch A~ to FP64 rounding;
  * the preconditioner: rank, sigma(A~), sigma(AN) (Lemma 4.3: both equal
    1/sigma(GU) for the same G), and range(N);
  * the solution: ||x - x*|| <= 1e-10 ||x*|| against the refined min-length
    solution, and ||A^T r|| / (||A|| ||r||) <= 1e-12 with r, A^T r in
    double-double; iteration counts as the oracle's LSRN with the same G.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")

TOL_X = 1e-10          # relative error target
TOL_NE = 1e-12         # normal-equation residual target


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _ne_resid(A, b, x):
    r = O.dd_residual(A, b, x)
    g = O.dd_atr(A, r)
    return np.linalg.norm(g) / (O.two_norm_estimate(A) * np.linalg.norm(r))


@pytest.mark.parametrize("seed,tag,i0,j0,rows,cols", [
    (0, 0, 0, 0, 64, 128), (12345, 0, 17, 3, 33, 61), (2 ** 40 + 7, 1, 999_983, 5, 5, 37),
    (9, 0, 123, 2 ** 32 - 3, 4, 9)])
def test_sketch_matrix_bitwise(seed, tag, i0, j0, rows, cols):
    g, z = L.lsrn_generate_sketch_block(seed, tag, i0, j0, rows, cols, with_normals=True)
    assert np.array_equal(z, O.normals(seed, tag, i0, j0, rows, cols))
    assert np.array_equal(g, O.sketch_block(seed, i0, j0, rows, cols, tag=tag))


def test_sketch_matrix_bitwise_many():
    g = L.lsrn_generate_sketch_block(5, 0, 0, 0, 2000, 500)
    assert np.array_equal(g, O.sketch_block(5, 0, 0, 2000, 500))


def _oracle_sketch(A, seed, gamma=2.0, lam=0.0):
    m, n = A.shape
    if m >= n:
        B = np.vstack([A, lam * np.eye(n)]) if lam > 0 else A
        s = math.ceil(gamma * n)
        return O.sketch_block(seed, 0, 0, B.shape[0], s).T @ B
    B = np.hstack([A / lam, np.eye(m)]) if lam > 0 else A
    s = math.ceil(gamma * m)
    return (B @ O.sketch_block(seed, 0, 0, B.shape[1], s)).T


@pytest.mark.parametrize("m,n,lam", [(2000, 100, 0.0), (777, 37, 0.0), (300, 1, 0.0),
                                     (37, 777, 0.0), (501, 64, 0.3), (40, 450, 0.2),
                                     (130, 129, 0.0)])
def test_sketch_parity(m, n, lam):
    rng = np.random.Generator(np.random.PCG64(m * 7 + n))
    A = rng.standard_normal((m, n))
    plan = L.lsrn_plan(_dev(A), L.default_options(seed=11, lambda_=lam))
    L.lsrn_sketch(plan)
    S = L.lsrn_plan_get_sketch(plan)
    ref = _oracle_sketch(A, 11, lam=lam)
    assert S.shape == ref.shape
    assert np.linalg.norm(S - ref) <= 1e-13 * np.linalg.norm(ref)


def test_preconditioner_parity_c1():
    P = W.c1_problem(0)
    plan = L.lsrn_plan(_dev(P.A), L.default_options(seed=0))
    L.lsrn_sketch(plan)
    r = L.lsrn_precond(plan)
    N, sig = L.lsrn_plan_get_precond(plan)
    _, info = O.lsrn(P.A, P.b, seed=0, max_iter=1)
    assert r == info["rank"] == 80
    assert np.allclose(sig, info["sigma_sketch"][:r], rtol=1e-10)
    # Lemma 4.3: sigma(AN) = 1 / sigma(G U) for the same G -- for both N's
    s = info["s"]
    G = O.sketch_block(0, 0, 0, P.A.shape[0], s).T
    ref = np.sort(1.0 / np.linalg.svd(G @ P.meta["U"], compute_uv=False))
    got = np.sort(np.linalg.svd(P.A @ N, compute_uv=False))
    assert np.allclose(got, ref, rtol=1e-7)
    # range(N) = range(N_oracle)
    No = info["N"]
    Q, _ = np.linalg.qr(No)
    assert np.linalg.norm(N - Q @ (Q.T @ N)) <= 1e-9 * np.linalg.norm(N)


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_solve_c1(solver):
    P = W.c1_problem(0)
    xs, _ = O.minlen_refined(P.A, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), solver=solver, seed=0)
    x = x.cpu().numpy()
    assert info["rank"] == 80 and info["s"] == 200
    assert O.rel_err(x, xs) <= TOL_X
    assert _ne_resid(P.A, P.b, x) <= TOL_NE
    xo, io = O.lsrn(P.A, P.b, solver=solver, seed=0, refine=1)
    if solver == "lsqr":
        assert abs(info["iterations"] - io["iterations"]) <= 1
    else:
        assert info["iterations"] == io["iterations"]
    assert info["refine_iterations"] == io["refine_steps"][0]
    # the GPU and the oracle's LSRN agree to the FP64 floor
    assert O.rel_err(x, xo) <= TOL_X


def test_solve_without_refinement_matches_oracle_lsrn():
    P = W.c1_problem(0)
    x, info = L.solve(_dev(P.A), _dev(P.b), solver="lsqr", seed=3, refine_max=0)
    xo, io = O.lsrn(P.A, P.b, solver="lsqr", seed=3)
    assert abs(info["iterations"] - io["iterations"]) <= 1
    assert O.rel_err(x.cpu().numpy(), xo) <= 1e-9
    assert info["rnorm_est"] == pytest.approx(io["lsqr"]["rnorm"], rel=1e-8)


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_solve_fat_rank_deficient(solver):
    P = W.dense_haar(1500, 70, 55, 1e5, 0.0, seed=4)
    A = np.ascontiguousarray(P.A.T)                   # 70 x 1500, rank 55
    b = A @ np.random.Generator(np.random.PCG64(5)).standard_normal(1500)
    xs, _ = O.minlen_refined(A, b)
    x, info = L.solve(_dev(A), _dev(b), solver=solver, seed=1)
    assert info["tall"] == 0 and info["rank"] == 55
    assert O.rel_err(x.cpu().numpy(), xs) <= TOL_X


@pytest.mark.parametrize("shape", [(900, 40), (40, 900)])
@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_ridge(shape, solver):
    rng = np.random.Generator(np.random.PCG64(sum(shape)))
    A = rng.standard_normal(shape)
    b = rng.standard_normal(shape[0])
    lam = 1e-2
    x, info = L.solve(_dev(A), _dev(b), solver=solver, lambda_=lam, seed=2)
    ref = O.ridge_closed_form(A, b, lam)
    assert O.rel_err(x.cpu().numpy(), ref) <= TOL_X
    xo, _ = O.lsrn(A, b, solver=solver, lam=lam, seed=2, refine=1)
    assert O.rel_err(x.cpu().numpy(), xo) <= TOL_X


def test_host_pointers_layouts_and_f32():
    P = W.dense_haar(640, 48, 48, 1e3, 1e-3, seed=9)
    xs, _ = O.minlen_refined(P.A, P.b)
    # host arrays in and out
    x, _ = L.solve(P.A, P.b, seed=4)
    assert isinstance(x, np.ndarray) and O.rel_err(x, xs) <= TOL_X
    # column-major storage (the plan transposes it on the device)
    At = np.ascontiguousarray(P.A.T)
    x2, _ = L.solve(_dev(At), _dev(P.b), layout="col", seed=4)
    assert O.rel_err(x2.cpu().numpy(), xs) <= TOL_X
    # padded leading dimension
    Ap = np.zeros((640, 51))
    Ap[:, :48] = P.A
    x3, _ = L.solve(_dev(Ap)[:, :48], _dev(P.b), seed=4)
    assert O.rel_err(x3.cpu().numpy(), xs) <= TOL_X
    # float32 storage: the solution of the rounded matrix
    A32 = P.A.astype(np.float32)
    x4, _ = L.solve(_dev(A32), _dev(P.b), seed=4)
    xs32, _ = O.minlen_refined(A32.astype(np.float64), P.b)
    assert O.rel_err(x4.cpu().numpy(), xs32) <= TOL_X


@pytest.mark.parametrize("m,n", [(1, 1), (5, 1), (1, 6), (64, 64), (2049, 33), (33, 2049),
                                 (3000, 513), (1025, 1025)])
def test_ragged_and_square_shapes(m, n):
    rng = np.random.Generator(np.random.PCG64(m + 1000 * n))
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    xs = O.minlen_svd(A, b)
    x, info = L.solve(_dev(A), _dev(b), seed=0)
    assert info["rank"] == min(m, n)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-9


def test_zero_matrix_and_zero_rhs():
    A = np.zeros((50, 6))
    x, info = L.solve(_dev(A), _dev(np.ones(50)), seed=0)
    assert info["rank"] == 0 and torch.count_nonzero(x).item() == 0
    B = np.random.Generator(np.random.PCG64(1)).standard_normal((50, 6))
    x, info = L.solve(_dev(B), _dev(np.zeros(50)), seed=0)
    assert torch.count_nonzero(x).item() == 0


def test_invalid_arguments_and_state():
    A = _dev(np.ones((10, 3)))
    for kw in (dict(gamma=1.0), dict(lambda_=-1.0), dict(tol=0.0), dict(refine_max=-1)):
        with pytest.raises(L.LsrnError) as e:
            L.lsrn_plan(A, L.default_options(**kw))
        assert e.value.status == L.LSRN_ERR_INVALID_ARG
    plan = L.lsrn_plan(A)
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_precond(plan)
    assert e.value.status == L.LSRN_ERR_STATE


def test_cs_invalid_when_bounds_do_not_exist():
    # gamma close to 1 and full rank: (1 - 1/sqrt(s)) sqrt(s) <= sqrt(r)
    rng = np.random.Generator(np.random.PCG64(3))
    A = _dev(rng.standard_normal((400, 20)))
    with pytest.raises(L.LsrnError) as e:
        L.solve(A, _dev(rng.standard_normal(400)), solver="cs", gamma=1.01)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG


def test_plan_reuse_many_rhs():
    P = W.c1_problem(0)
    plan = L.lsrn_plan(_dev(P.A), L.default_options(seed=0))
    rng = np.random.Generator(np.random.PCG64(8))
    for k in range(3):
        b = P.A @ rng.standard_normal(100) + 1e-3 * rng.standard_normal(2000)
        xs, _ = O.minlen_refined(P.A, b)
        x, _ = L.lsrn_solve_lsqr(plan, _dev(b))
        assert O.rel_err(x.cpu().numpy(), xs) <= TOL_X
    plan.close()


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_tall_householder_medium(solver):
    # the 10^6 x 2000 recipe at 1/20 of the rows and 1/10 of the columns
    P = W.dense_householder(50_000, 200, 180, 1e6, 1e-4, seed=1)
    xs, _ = O.minlen_refined(P.A, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), solver=solver, seed=0)
    assert info["rank"] == 180 and info["s"] == 400
    assert O.rel_err(x.cpu().numpy(), xs) <= TOL_X
    assert _ne_resid(P.A, P.b, x.cpu().numpy()) <= TOL_NE
    xf = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    assert O.rel_err(x.cpu().numpy(), xf) <= 1e-8      # planted factors: data-rounding floor
