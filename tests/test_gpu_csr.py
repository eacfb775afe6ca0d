"""GPU parity of the sparse (CSR) path against the oracle: the sketch A~ = G A
or A G formed from the sparse columns, and full solves for m >= n and m < n,
with and without Tikhonov regularisation (section 5), on sprandn-like and
fixed-nnz-per-row matrices (section 6.5)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _csr_args(C, device=True, dtype=np.float64):
    conv = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")) if device else np.ascontiguousarray
    return (C.m, C.n, conv(C.row_ptr), conv(C.col_idx), conv(C.values.astype(dtype)))


def _oracle_sketch(D, seed, lam=0.0):
    m, n = D.shape
    if m >= n:
        B = np.vstack([D, lam * np.eye(n)]) if lam > 0 else D
        return O.sketch_block(seed, 0, 0, B.shape[0], math.ceil(2 * n)).T @ B
    B = np.hstack([D / lam, np.eye(m)]) if lam > 0 else D
    return (B @ O.sketch_block(seed, 0, 0, B.shape[1], math.ceil(2 * m))).T


@pytest.mark.parametrize("m,n,dens,lam", [(3000, 80, 0.05, 0.0), (60, 4000, 0.02, 0.0),
                                          (1500, 40, 0.1, 0.5), (50, 3000, 0.03, 1e-3)])
def test_csr_sketch_parity(m, n, dens, lam):
    C = W.csr_random_density(m, n, dens, seed=m + n)
    plan = L.lsrn_plan(None, L.default_options(seed=4, lambda_=lam), csr=_csr_args(C))
    L.lsrn_sketch(plan)
    S = L.lsrn_plan_get_sketch(plan)
    plan.close()
    ref = _oracle_sketch(C.to_dense(), 4, lam)
    assert np.linalg.norm(S - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
def test_csr_tall(solver):
    C = W.csr_random_density(4000, 100, 0.05, seed=11)
    D = C.to_dense()
    b = np.random.Generator(np.random.PCG64(12)).standard_normal(4000)
    x, info = L.solve(None, _dev(b), solver=solver, csr=_csr_args(C), seed=1)
    assert info["tall"] == 1 and info["rank"] == 100
    assert O.rel_err(x.cpu().numpy(), O.minlen_svd(D, b)) <= 1e-10


@pytest.mark.parametrize("solver", ["lsqr", "cs"])
@pytest.mark.parametrize("lam", [0.0, 1e-3])
def test_csr_fat_uniform_rows(solver, lam):
    # the 10^4 x 10^6, 2000 nnz/row recipe scaled to 200 x 20000, 40 nnz/row
    C = W.csr_uniform_rows(200, 20000, 40, seed=5)
    D = C.to_dense()
    b = W.gaussian_vector(200, 6)
    x, info = L.solve(None, _dev(b), solver=solver, csr=_csr_args(C), seed=3, lambda_=lam)
    ref = O.ridge_closed_form(sp.csr_matrix(D), b, lam) if lam > 0 else O.minlen_svd(D, b)
    assert info["tall"] == 0
    assert O.rel_err(x.cpu().numpy(), ref) <= 1e-10


def test_csr_f32_values_and_host_arrays():
    C = W.csr_uniform_rows(150, 9000, 30, seed=8, dtype=np.float32)
    D = C.to_dense()
    b = W.gaussian_vector(150, 9)
    x, _ = L.solve(None, b, csr=_csr_args(C, device=False, dtype=np.float32), seed=2)
    assert isinstance(x, np.ndarray)
    assert O.rel_err(x, O.minlen_svd(D, b)) <= 1e-10


def test_csr_rank_deficient_tall():
    rng = np.random.Generator(np.random.PCG64(3))
    D = sp.random(2000, 60, density=0.1, random_state=3, format="csr").toarray()
    D[:, 50:] = D[:, :10] @ rng.standard_normal((10, 10))       # rank 50
    C = sp.csr_matrix(D)
    C.sort_indices()
    args = (2000, 60, _dev(C.indptr.astype(np.int64)), _dev(C.indices.astype(np.int32)),
            _dev(C.data))
    b = rng.standard_normal(2000)
    x, info = L.solve(None, _dev(b), csr=args, seed=5)
    assert info["rank"] == 50
    assert O.rel_err(x.cpu().numpy(), O.minlen_svd(D, b, rcond=1e-12)) <= 1e-10


def test_csr_invalid_structure():
    C = W.csr_uniform_rows(20, 100, 5, seed=1)
    bad_col = C.col_idx.copy()
    bad_col[7] = 100
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_plan(None, csr=(20, 100, _dev(C.row_ptr), _dev(bad_col), _dev(C.values)))
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
    bad_rp = C.row_ptr.copy()
    bad_rp[5], bad_rp[6] = bad_rp[6], bad_rp[5]
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_plan(None, csr=(20, 100, _dev(bad_rp), _dev(C.col_idx), _dev(C.values)))
    assert e.value.status == L.LSRN_ERR_INVALID_ARG


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
