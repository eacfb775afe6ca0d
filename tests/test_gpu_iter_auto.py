"""LSRN_ITER_AUTO: the pass precision is chosen by the size of A (FP64 below
1 GiB of FP64 entries and for CSR; above it the double-float planes where
they apply, FP32 for tall A with a short side <= 512).  Whatever the choice,
the solve meets the FP64 path's accuracy against the reference."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def test_small_dense_and_csr_run_fp64_passes():
    P = W.dense_householder(20_000, 300, 280, 1e5, 1e-4, seed=21)
    xs = O.minlen_from_factors(P.apply_Ut, P.sigma, P.apply_V, P.b)
    x, info = L.solve(_dev(P.A), _dev(P.b), seed=2, iter_mode=L.LSRN_ITER_AUTO,
                      sketch_mode=L.LSRN_SKETCH_TC_SLICED)
    assert info["iter_used"] == L.LSRN_ITER_F64
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10
    C = W.csr_sprandn(3000, 200, 0.05, seed=4)
    b = np.random.default_rng(5).standard_normal(3000)
    csr = (C.m, C.n, _dev(C.row_ptr), _dev(C.col_idx), _dev(C.values))
    x, info = L.solve(None, _dev(b), csr=csr, seed=2, iter_mode=L.LSRN_ITER_AUTO)
    assert info["iter_used"] == L.LSRN_ITER_F64
    ref = O.minlen_svd(C.to_dense(), b)
    assert O.rel_err(x.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("m,n,expect", [(70_000, 2000, "x2"), (300_000, 480, "f32")])
def test_large_tall_dense_take_the_reduced_precision_passes(m, n, expect):
    rng = np.random.default_rng(m % 1000)
    A = rng.standard_normal((m, n))
    A[:, 7] *= 1e-4                          # some spread in the column scales
    b = rng.standard_normal(m)
    Ad, bd = _dev(A), _dev(b)
    x, info = L.solve(Ad, bd, seed=9, iter_mode=L.LSRN_ITER_AUTO, sketch_mode=L.LSRN_SKETCH_TC_SLICED)
    want = L.LSRN_ITER_F32X2 if expect == "x2" else L.LSRN_ITER_F32
    assert info["iter_used"] == want
    x64, i64 = L.solve(Ad, bd, seed=9, iter_mode=L.LSRN_ITER_F64, sketch_mode=L.LSRN_SKETCH_TC_SLICED)
    assert i64["iter_used"] == L.LSRN_ITER_F64
    x, x64 = x.cpu().numpy(), x64.cpu().numpy()
    assert O.rel_err(x, x64) <= 1e-10
    # normal equations in double-double on the host, relative to ||A||_2 ||r||
    r = O.dd_residual(A, b, x)
    ne = np.linalg.norm(O.dd_atr(A, r)) / (O.two_norm_estimate(A) * np.linalg.norm(r))
    assert ne <= 1e-12
