"""The FP32 planes of the double-float passes (LSRN_ITER_F32X2) are the three-way
round-to-nearest split of X' = X / 2^e, X = A (m >= n) or A^T (m < n) and 2^e
the power of two that puts max |X| in [1, 2): hi = fl32(X'), lo = fl32(X' - hi),
x3 = fl32(X' - hi - lo), zero in the padding columns.  Checked bit for bit
against the same split done with numpy's IEEE casts, on matrices that reach
the rounding ties, the carry into the next binade, signed zeros, subnormals,
entries far below the largest one, both paths of the conversion (rows of whole
column pairs and odd short sides) and scales near both ends of the double
range."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _split(X):
    """The definition: scale by the power of two, then round to nearest three times."""
    mx = float(np.max(np.abs(X))) if X.size else 0.0
    scale = 1.0
    if mx > 0.0 and math.isfinite(mx):
        scale = math.ldexp(1.0, math.frexp(mx)[1] - 1)
    V = X * (1.0 / scale)
    h = V.astype(np.float32)
    r = V - h.astype(np.float64)
    lo = r.astype(np.float32)
    x3 = (r - lo.astype(np.float64)).astype(np.float32)
    return h, lo, x3, scale


def _planes(A):
    plan = L.lsrn_plan(torch.from_numpy(np.ascontiguousarray(A)).to("cuda"),
                       L.default_options(seed=5, iter_mode=L.LSRN_ITER_F32X2))
    try:
        return L.lsrn_plan_get_planes(plan)
    finally:
        plan.close()


def _check(A):
    X = A if A.shape[0] >= A.shape[1] else A.T
    hi, lo, x3, scale = _planes(A)
    eh, el, e3, escale = _split(X)
    q = X.shape[1]
    assert hi.shape[0] == X.shape[0] and hi.shape[1] == (q + 3) // 4 * 4
    assert scale == escale
    for got, want in ((hi, eh), (lo, el), (x3, e3)):
        assert np.array_equal(got[:, :q].view(np.uint32), want.view(np.uint32))
        assert not np.any(got[:, q:].view(np.uint32))


def _ties_and_edges(m, n, seed):
    """Entries M 2^(E-52) with the low 29 significand bits at and around the
    rounding tie (2^28), all ones, zero; top 24 bits all ones (carry); E from
    -110 to 0 so that some entries leave the normal range of the lower planes;
    plus signed zeros, subnormals and the smallest normal double."""
    rng = np.random.default_rng(seed)
    top = rng.integers(1 << 23, 1 << 24, size=(m, n), dtype=np.int64)
    top[rng.random((m, n)) < 0.05] = (1 << 24) - 1
    rems = np.array([1 << 28, (1 << 28) + 1, (1 << 28) - 1, (1 << 29) - 1, 0, 1], dtype=np.int64)
    rem = np.where(rng.random((m, n)) < 0.6, rems[rng.integers(0, len(rems), size=(m, n))],
                   rng.integers(0, 1 << 29, size=(m, n), dtype=np.int64))
    M = (top << 29) | rem
    E = rng.integers(-110, 1, size=(m, n))
    A = np.ldexp(M.astype(np.float64), (E - 52).astype(np.int32))   # M < 2^53: exact
    A *= np.where(rng.random((m, n)) < 0.5, -1.0, 1.0)
    A[0, 0] = 1.75                       # every entry is below 2: scale 1
    specials = [0.0, -0.0, 5e-324, -2.5e-320, 2.2250738585072014e-308, -1e-300]
    for k, v in enumerate(specials):
        A[1 + k, k] = v
    return A


@pytest.mark.parametrize("m,n", [(4001, 600), (3001, 513), (2000, 1031)])
def test_planes_gaussian(m, n):
    A = np.random.default_rng(m).standard_normal((m, n))
    _check(A)


def test_planes_fat_orientation():
    _check(np.random.default_rng(7).standard_normal((600, 5000)))


@pytest.mark.parametrize("n", [1024, 1031])
def test_planes_ties_carries_and_special_values(n):
    _check(_ties_and_edges(3000, n, seed=n))


@pytest.mark.parametrize("scale", [2.0 ** -300, 3e80, 2.0 ** 1000, 1e-305])
def test_planes_extreme_scales(scale):
    _check(np.random.default_rng(11).standard_normal((2500, 700)) * scale)


def test_planes_zero_matrix_and_unsupported_modes():
    _check(np.zeros((1500, 600)))
    A = torch.from_numpy(np.random.default_rng(3).standard_normal((1500, 600))).to("cuda")
    plan = L.lsrn_plan(A, L.default_options(seed=5, iter_mode=L.LSRN_ITER_F64))
    try:
        with pytest.raises(L.LsrnError):
            L.lsrn_plan_get_planes(plan)
    finally:
        plan.close()
