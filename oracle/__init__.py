"""LSRN oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 CPU restatement of what the paper computes, used to judge
the CUDA path.  Only the tests, the smoke check (``__graft_entry__.smoke``) and
the CPU-baseline leg of ``bench.py`` import this package; the product library
never does, and this package shares no code with it (the CUDA sources are not
read, linked or imported here).  Library primitives (numpy matmul, LAPACK QR /
Cholesky / triangular solves through numpy and scipy) serve as single steps;
everything else follows the paper's notation in the paper's order.

Sections of the paper followed here:
  * section 1, eqs. (ls), (ls_min_length): the min-length least-squares
    solution x* of min ||Ax - b||_2                        -> ``minlen_svd``
  * section 2.1: x* = V Sigma^-1 U^T b (SVD route), x* = Z T^-1 Q^T b
    (complete orthogonal factorisation)                    -> ``minlen_svd``,
    ``minlen_cod``, ``minlen_from_factors``
  * section 4.1, Algorithm 1 (m >> n) and Algorithm 2 (m << n)   -> ``lsrn``
  * section 4.2, Theorem 4.5 (bounds on sigma(AN)) and Theorem 4.6 (iteration
    count)                                                 -> ``thm45_bounds``,
    ``thm46_bound``
  * section 4.2, Algorithm 3 (Chebyshev semi-iterative method) -> ``chebyshev``
  * section 5, eqs. (l2_reg_eq) and (l2_reg_eq_under): Tikhonov regularisation
    with W = lambda I by augmentation                      -> ``lsrn(lam=...)``,
    ``ridge_closed_form``
  * LSQR is the algorithm of Paige and Saunders (ACM TOMS 8(1), 1982), which the
    paper cites and uses but does not print              -> ``lsqr``

Readings of the paper that the oracle takes:
  * Algorithm 3, k = 1: alpha = 1 / (d - c^2 / (2 d)) (the printed formula lacks
    the reciprocal; only this reading reproduces the Chebyshev polynomial
    residual, which a test pins).
  * Algorithm 3 loop: k = 0..K inclusive, K = ceil((log eps - log 2) / log rho),
    rho = (sigma_U - sigma_L) / (sigma_U + sigma_L); for k >= 2 beta uses the
    previous alpha, then alpha is updated.
  * Theorem 4.5 bounds used by Algorithm 3 inside LSRN: sigma_U =
    1/((1-a) sqrt(s) - sqrt(r)), sigma_L = 1/((1+a) sqrt(s) + sqrt(r)) with
    a = 1/sqrt(s) by default (t = 1 in Lemma 4.4); this reproduces the 106
    Chebyshev iterations of Table 3.
  * r = rank(A~) is the numerical rank #{sigma_i > rcond * sigma_1}, rcond
    defaulting to max(s, n) * 2^-53 (max(m, n) * 2^-53 for x*).
  * G's entries are the Box-Muller normals rounded to the grid 2^-12, drawn as
    Gamma[long-side index, sketch index]; G = Gamma^T (m >= n) or Gamma (m < n).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Callable, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsrn_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblsrn_oracle.so")

TAG_SKETCH = 0          # Philox tag of the sketching matrix G
EPS64 = 2.0 ** -53


# --------------------------------------------------------------------------- #
# Build / load the C part                                                     #
# --------------------------------------------------------------------------- #
def build(force: bool = False) -> str:
    """Compile lsrn_oracle.c (plain C, -ffp-contract=off) into _build/."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.orc_uniform.argtypes = [ctypes.c_uint32]
        lib.orc_uniform.restype = ctypes.c_float
        lib.orc_logf.argtypes = [ctypes.c_float]
        lib.orc_logf.restype = ctypes.c_float
        lib.orc_sincos2pi.argtypes = [ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_float)]
        lib.orc_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                   ctypes.c_uint64]
        lib.orc_normal.restype = ctypes.c_float
        lib.orc_sketch_entry.argtypes = lib.orc_normal.argtypes
        lib.orc_sketch_entry.restype = ctypes.c_float
        lib.orc_gauss_block.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_jacobi_svd.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        lib.orc_jacobi_svd.restype = ctypes.c_int
        lib.orc_dd_residual.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
        lib.orc_dd_atr.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        _lib_handle = lib
    return _lib_handle


# --------------------------------------------------------------------------- #
# Random sketching matrix (Algorithms 1, 2 step 2)                             #
# --------------------------------------------------------------------------- #
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (ctypes.c_uint32 * 4)()
    _lib().orc_philox4x32_10(c, k, out)
    return tuple(int(v) for v in out)


def uniform(x: int) -> float:
    return _lib().orc_uniform(int(x) & 0xFFFFFFFF)


def logf(u: float) -> float:
    return _lib().orc_logf(float(u))


def sincos2pi(u: float):
    s, c = ctypes.c_float(), ctypes.c_float()
    _lib().orc_sincos2pi(float(u), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def normal_at(seed: int, tag: int, i: int, j: int) -> float:
    return _lib().orc_normal(seed, tag, i, j)


def normals(seed: int, tag: int, i0: int, j0: int, rows: int, cols: int) -> np.ndarray:
    """Box-Muller normals z[i0:i0+rows, j0:j0+cols] (float32)."""
    z = np.empty((rows, cols), dtype=np.float32)
    _lib().orc_gauss_block(seed, tag, i0, j0, rows, cols, z.ctypes.data, None)
    return z


def sketch_block(seed: int, i0: int, j0: int, rows: int, cols: int,
                 tag: int = TAG_SKETCH) -> np.ndarray:
    """Entries [i0:i0+rows, j0:j0+cols] of the drawing array Gamma of the
    sketching matrix (float64): Gamma[l, i] is the draw for long-side index l
    (row of A for m >= n, column of A for m < n) and sketch index i < s, so one
    Philox call covers four consecutive sketch indices.  Algorithm 1 uses
    G = Gamma^T (s x m), Algorithm 2 uses G = Gamma (n x s)."""
    g = np.empty((rows, cols), dtype=np.float64)
    _lib().orc_gauss_block(seed, tag, i0, j0, rows, cols, None, g.ctypes.data)
    return g


# --------------------------------------------------------------------------- #
# SVD (one-sided Jacobi in C) and min-length solutions (section 2.1)           #
# --------------------------------------------------------------------------- #
def jacobi_svd(X: np.ndarray, tol: Optional[float] = None, max_sweeps: int = 60):
    """Thin SVD X = U diag(sigma) V^T by one-sided Jacobi, sigma descending.

    For p >= q the columns of X are rotated; for p < q the method is applied to
    X^T and the factors are swapped.  U's columns for zero singular values are
    left as zero vectors (they are never used).
    """
    X = np.asarray(X, dtype=np.float64)
    p, q = X.shape
    if p < q:
        U, s, V = jacobi_svd(X.T, tol, max_sweeps)
        return V, s, U
    if tol is None:
        tol = p * EPS64
    W = np.asfortranarray(X.copy())
    V = np.zeros((q, q), order="F")
    sig = np.zeros(q)
    sweeps = _lib().orc_jacobi_svd(p, q, W.ctypes.data, p, V.ctypes.data, q, sig.ctypes.data,
                                   tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("one-sided Jacobi did not converge")
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    W = W[:, order]
    V = np.ascontiguousarray(V[:, order])
    U = np.zeros_like(W)
    nz = sig > 0
    U[:, nz] = W[:, nz] / sig[nz]
    return np.ascontiguousarray(U), sig, V


def numerical_rank(sigma: np.ndarray, rcond: float) -> int:
    if sigma.size == 0 or sigma[0] == 0.0:
        return 0
    return int(np.count_nonzero(sigma > rcond * sigma[0]))


def default_rcond(p: int, q: int) -> float:
    return max(p, q) * EPS64


def minlen_svd(A: np.ndarray, b: np.ndarray, rcond: Optional[float] = None) -> np.ndarray:
    """x* = V_r Sigma_r^-1 U_r^T b over the singular values above rcond * sigma_1."""
    A = np.asarray(A, dtype=np.float64)
    if rcond is None:
        rcond = default_rcond(*A.shape)
    U, s, V = jacobi_svd(A)
    r = numerical_rank(s, rcond)
    return V[:, :r] @ ((U[:, :r].T @ b) / s[:r])


def pinv_svd(A: np.ndarray, rcond: Optional[float] = None) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    if rcond is None:
        rcond = default_rcond(*A.shape)
    U, s, V = jacobi_svd(A)
    r = numerical_rank(s, rcond)
    return (V[:, :r] / s[:r]) @ U[:, :r].T


def minlen_cod(A: np.ndarray, b: np.ndarray, rcond: Optional[float] = None) -> np.ndarray:
    """x* by a complete orthogonal factorisation A P = Q [T^T 0] Z^T (section 2.1).

    Column-pivoted QR gives A P = Q R; the leading k rows of R (k = numerical
    rank from |R_ii|) are factored as R_k = T^T Z^T by a QR of R_k^T; then
    x*[P] = Z T^-T Q_k^T b.
    """
    import scipy.linalg as sla
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if rcond is None:
        rcond = default_rcond(m, n)
    Q, R, P = sla.qr(A, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    k = int(np.count_nonzero(d > rcond * d[0])) if d.size and d[0] > 0 else 0
    x = np.zeros(n)
    if k == 0:
        return x
    Z, T = np.linalg.qr(R[:k, :].T)
    y = sla.solve_triangular(T.T, Q[:, :k].T @ b, lower=True)
    x[P] = Z @ y
    return x


def dd_residual(A: np.ndarray, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """r = b - A x accumulated in double-double, rounded to FP64 (dense row-major A)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.empty(A.shape[0])
    _lib().orc_dd_residual(A.shape[0], A.shape[1], A.ctypes.data, A.shape[1], b.ctypes.data,
                           x.ctypes.data, r.ctypes.data)
    return r


def dd_atr(A: np.ndarray, r: np.ndarray) -> np.ndarray:
    """g = A^T r accumulated in double-double, rounded to FP64 (dense row-major A)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    g = np.empty(A.shape[1])
    _lib().orc_dd_atr(A.shape[0], A.shape[1], A.ctypes.data, A.shape[1], r.ctypes.data,
                      g.ctypes.data)
    return g


def minlen_refined(A: np.ndarray, b: np.ndarray, rcond: Optional[float] = None,
                   steps: int = 3):
    """x* of the stored A below the FP64 floor: start from the SVD solution and
    apply corrected-seminormal steps x <- x + V_r Sigma_r^-2 V_r^T A^T(b - A x),
    with r = b - A x and A^T r both accumulated in double-double (the
    correction solves A^T A d = A^T r on range(A^T), the normal equation whose
    solution set section 2.1 characterises).  Returns (x, norms of corrections)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    if rcond is None:
        rcond = default_rcond(*A.shape)
    U, s, V = jacobi_svd(A)
    r = numerical_rank(s, rcond)
    Vr, sr = V[:, :r], s[:r]
    x = Vr @ ((U[:, :r].T @ b) / sr)
    corr = []
    for _ in range(steps):
        res = dd_residual(A, b, x)
        g = dd_atr(A, res)
        d = Vr @ ((Vr.T @ g) / (sr * sr))
        x = x + d
        corr.append(float(np.linalg.norm(d)))
    return x, corr


def minlen_from_factors(apply_Ut: Callable, sigma: np.ndarray, apply_V: Callable,
                        b: np.ndarray) -> np.ndarray:
    """x* = V Sigma^-1 U^T b with the factors the generator planted (section 2.1)."""
    return apply_V(apply_Ut(b) / sigma)


def ridge_closed_form(A, b: np.ndarray, lam: float) -> np.ndarray:
    """argmin 1/2||Ax-b||^2 + 1/2||lam x||^2 by Cholesky of the regularised normal
    equations (section 5, W = lam I): (A^T A + lam^2 I)^-1 A^T b when m >= n,
    A^T (A A^T + lam^2 I)^-1 b when m < n.  A may be dense or scipy.sparse."""
    import scipy.linalg as sla
    m, n = A.shape
    if m >= n:
        K = A.T @ A
        K = np.asarray(K.todense()) if hasattr(K, "todense") else np.asarray(K)
        K = K + lam * lam * np.eye(n)
        c = sla.cho_factor(K, lower=True)
        return sla.cho_solve(c, np.asarray(A.T @ b).ravel())
    K = A @ A.T
    K = np.asarray(K.todense()) if hasattr(K, "todense") else np.asarray(K)
    K = K + lam * lam * np.eye(m)
    c = sla.cho_factor(K, lower=True)
    return np.asarray(A.T @ sla.cho_solve(c, b)).ravel()


# --------------------------------------------------------------------------- #
# Iterative solvers                                                            #
# --------------------------------------------------------------------------- #
def lsqr(matvec: Callable, rmatvec: Callable, b: np.ndarray, n: int, atol: float = 1e-14,
         btol: float = 1e-14, iter_lim: int = 1000):
    """LSQR of Paige and Saunders (1982): Golub-Kahan bidiagonalisation of the
    operator with the QR update of the bidiagonal, x_0 = 0.

    Stopping rules S1 (||r|| <= btol ||b|| + atol ||A|| ||x||) and S2
    (||A^T r|| <= atol ||A|| ||r||) with the estimates ||r_k|| = phibar_{k+1},
    ||A^T r_k|| = phibar_{k+1} alpha_{k+1} |c_k| and ||A|| estimated by the
    Frobenius norm of the bidiagonal; ||x_k|| is computed directly.
    Returns (x, info) with info['history'] = [(rnorm, arnorm) per iteration].
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n)
    info = dict(istop=0, itn=0, history=[], anorm=0.0, rnorm=0.0, arnorm=0.0)
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return x, info
    u = b / beta
    v = rmatvec(u)
    alpha = float(np.linalg.norm(v))
    info["rnorm"] = beta
    if alpha == 0.0:
        return x, info
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    bnorm = beta
    anorm2 = 0.0
    for itn in range(1, iter_lim + 1):
        u = matvec(v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
        anorm2 += alpha * alpha + beta * beta
        v = rmatvec(u) - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0.0:
            v = v / alpha
        rho = math.hypot(rhobar, beta)
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        rnorm = phibar
        arnorm = phibar * alpha * abs(c)
        anorm = math.sqrt(anorm2)
        xnorm = float(np.linalg.norm(x))
        info["history"].append((rnorm, arnorm))
        info.update(itn=itn, anorm=anorm, rnorm=rnorm, arnorm=arnorm)
        test1 = rnorm / bnorm
        test2 = arnorm / (anorm * rnorm) if anorm * rnorm > 0.0 else 0.0
        rtol = btol + atol * anorm * xnorm / bnorm
        if test1 <= rtol:
            info["istop"] = 1
            break
        if test2 <= atol:
            info["istop"] = 2
            break
        if alpha == 0.0 or beta == 0.0:
            info["istop"] = 3
            break
    return x, info


def cs_iteration_count(sigma_L: float, sigma_U: float, tol: float) -> int:
    """K in Algorithm 3's loop k = 0..K (K + 1 iterations)."""
    rho = (sigma_U - sigma_L) / (sigma_U + sigma_L)
    if rho <= 0.0:
        return 0
    return int(math.ceil((math.log(tol) - math.log(2.0)) / math.log(rho)))


def chebyshev(matvec: Callable, rmatvec: Callable, b: np.ndarray, n: int, sigma_L: float,
              sigma_U: float, tol: float = 1e-14):
    """Algorithm 3 (Chebyshev semi-iterative method) on min ||Bx - b||, x_0 = 0.

    d = (sU^2 + sL^2)/2, c = (sU^2 - sL^2)/2; for k = 0..K:
      beta = 0, (c/d)^2/2, (alpha c/2)^2;  alpha = 1/d, 1/(d - c^2/(2d)), 1/(d - alpha c^2/4)
      v <- beta v + B^T r;  x <- x + alpha v;  r <- r - alpha B v.
    """
    b = np.asarray(b, dtype=np.float64)
    d = 0.5 * (sigma_U * sigma_U + sigma_L * sigma_L)
    c = 0.5 * (sigma_U * sigma_U - sigma_L * sigma_L)
    K = cs_iteration_count(sigma_L, sigma_U, tol)
    x = np.zeros(n)
    v = np.zeros(n)
    r = b.copy()
    alpha = 0.0
    for k in range(K + 1):
        if k == 0:
            beta, alpha = 0.0, 1.0 / d
        elif k == 1:
            beta, alpha = 0.5 * (c / d) ** 2, 1.0 / (d - c * c / (2.0 * d))
        else:
            beta = (alpha * c / 2.0) ** 2
            alpha = 1.0 / (d - alpha * c * c / 4.0)
        v = beta * v + rmatvec(r)
        x = x + alpha * v
        r = r - alpha * matvec(v)
    return x, dict(iterations=K + 1, K=K, d=d, c=c)


def thm45_bounds(r: int, s: int, alpha: float):
    """Theorem 4.5: sigma(AN) lies in [1/((1+a)sqrt s + sqrt r), 1/((1-a)sqrt s - sqrt r)]
    with probability >= 1 - 2 exp(-a^2 s / 2).  Returns (sigma_L, sigma_U)."""
    lo = (1.0 - alpha) * math.sqrt(s) - math.sqrt(r)
    if lo <= 0.0:
        raise ValueError("Theorem 4.5 needs alpha < 1 - sqrt(r/s)")
    return 1.0 / ((1.0 + alpha) * math.sqrt(s) + math.sqrt(r)), 1.0 / lo


def thm45_kappa_bound(r: int, s: int, alpha: float) -> float:
    """Eq. (cond_concentration): kappa(AN) <= (1 + a + sqrt(r/s)) / (1 - a - sqrt(r/s))."""
    q = math.sqrt(r / s)
    return (1.0 + alpha + q) / (1.0 - alpha - q)


def thm46_bound(r: int, s: int, eps: float = 1e-14, alpha: float = 0.0) -> float:
    """Theorem 4.6: (log eps - log 2) / log(alpha + sqrt(r/s)) iterations."""
    return (math.log(eps) - math.log(2.0)) / math.log(alpha + math.sqrt(r / s))


def default_lsqr_cap(r: int, s: int, eps: float) -> int:
    if r == 0:
        return 1
    return int(math.ceil(1.5 * thm46_bound(r, s, eps)))


# --------------------------------------------------------------------------- #
# LSRN, Algorithms 1 and 2 (+ section 5 augmentation)                          #
# --------------------------------------------------------------------------- #
def _as_dense(A):
    if hasattr(A, "todense"):
        return np.asarray(A.todense(), dtype=np.float64)
    return np.asarray(A, dtype=np.float64)


def chebyshev_normal(apply_K: Callable, f: np.ndarray, sigma_L: float, sigma_U: float,
                     tol: float):
    """Algorithm 3's recurrence applied to the normal equations K z = f of a
    preconditioned operator B (K = B^T B, spectrum in [sL^2, sU^2]), carrying the
    normal-equation residual h = f - K z instead of B^T r.  Returns (z, steps)."""
    d = 0.5 * (sigma_U * sigma_U + sigma_L * sigma_L)
    c = 0.5 * (sigma_U * sigma_U - sigma_L * sigma_L)
    K = cs_iteration_count(sigma_L, sigma_U, tol)
    z = np.zeros_like(f)
    v = np.zeros_like(f)
    h = np.array(f, dtype=np.float64)
    alpha = 0.0
    for k in range(K + 1):
        if k == 0:
            beta, alpha = 0.0, 1.0 / d
        elif k == 1:
            beta, alpha = 0.5 * (c / d) ** 2, 1.0 / (d - c * c / (2.0 * d))
        else:
            beta = (alpha * c / 2.0) ** 2
            alpha = 1.0 / (d - alpha * c * c / 4.0)
        v = beta * v + h
        z = z + alpha * v
        h = h - alpha * apply_K(v)
    return z, K + 1


def lsrn(A, b, gamma: float = 2.0, seed: int = 0, solver: str = "lsqr", tol: float = 1e-14,
         lam: float = 0.0, rcond: Optional[float] = None, cs_alpha: Optional[float] = None,
         max_iter: Optional[int] = None, refine: int = 0, refine_tol: float = 1e-3):
    """Compute x ~= A^+ b by Algorithm 1 (m >= n) or Algorithm 2 (m < n).

    With lam > 0 the Tikhonov problem min ||Ax-b||^2 + ||lam x||^2 is solved by
    LSRN on [A; lam I] (m >= n, eq. l2_reg_eq) or on [A/lam, I_m] followed by
    x = z / lam (m < n, eq. l2_reg_eq_under).  A is dense (numpy) or a CSR
    object with row_ptr/col_idx/values (converted to dense here: the oracle is
    meant for sizes where that is cheap).
    With refine > 0, that many refinement steps follow the iteration (an
    addition to the paper, which stops at step 6): the residual r = b - B x and
    B^T r are accumulated in double-double; for m >= n the correction solves the
    preconditioned normal equations (N^T B^T B N) z = N^T B^T r with Algorithm
    3's recurrence to relative tolerance refine_tol and x += N z; for m < n it
    solves min ||M^T B d - M^T r|| with Algorithm 3 and x += d.
    Returns (x, info).
    """
    if hasattr(A, "row_ptr"):
        A = A.to_dense()
    A = _as_dense(A)
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    tall = m >= n
    info = dict(tall=tall)
    if tall:
        B = np.vstack([A, lam * np.eye(n)]) if lam > 0 else A
        rhs = np.concatenate([b, np.zeros(n)]) if lam > 0 else b
        s = int(math.ceil(gamma * n))
        G = sketch_block(seed, 0, 0, B.shape[0], s).T          # s x (m or m+n)
        At = G @ B                                              # s x n
        U_, sig, V_ = jacobi_svd(At)
        rc = default_rcond(s, n) if rcond is None else rcond
        r = numerical_rank(sig, rc)
        Nmat = V_[:, :r] / sig[:r]                              # n x r

        def matvec(y):
            return B @ (Nmat @ y)

        def rmatvec(u):
            return Nmat.T @ (B.T @ u)
        dim = r
    else:
        B = np.hstack([A / lam, np.eye(m)]) if lam > 0 else A
        rhs = b
        s = int(math.ceil(gamma * m))
        G = sketch_block(seed, 0, 0, B.shape[1], s)             # (n or n+m) x s
        At = B @ G                                              # m x s
        U_, sig, V_ = jacobi_svd(At)
        rc = default_rcond(s, m) if rcond is None else rcond
        r = numerical_rank(sig, rc)
        Mmat = U_[:, :r] / sig[:r]                              # m x r

        def matvec(xv):
            return Mmat.T @ (B @ xv)

        def rmatvec(t):
            return B.T @ (Mmat @ t)
        dim = B.shape[1]
        rhs = Mmat.T @ b
    info.update(s=s, rank=r, sigma_sketch=sig, sketch=At)
    if r == 0:
        x = np.zeros(n)
        info.update(iterations=0)
        return x, info
    if solver == "lsqr":
        cap = default_lsqr_cap(r, s, tol) if max_iter is None else max_iter
        sol, it = lsqr(matvec, rmatvec, rhs, dim, atol=tol, btol=tol, iter_lim=cap)
        info.update(iterations=it["itn"], istop=it["istop"], history=it["history"],
                    lsqr=it)
    elif solver == "cs":
        a = (1.0 / math.sqrt(s)) if cs_alpha is None else cs_alpha
        sL, sU = thm45_bounds(r, s, a)
        sol, it = chebyshev(matvec, rmatvec, rhs, dim, sL, sU, tol)
        info.update(iterations=it["iterations"], sigma_L=sL, sigma_U=sU)
    else:
        raise ValueError(solver)
    a = (1.0 / math.sqrt(s)) if cs_alpha is None else cs_alpha
    sL, sU = thm45_bounds(r, s, a) if refine > 0 else (0.0, 0.0)
    steps = []
    if tall:
        info["y"] = sol
        info["N"] = Nmat
        xf = Nmat @ sol
        for _ in range(refine):
            res = dd_residual(B, rhs, xf)
            g = dd_atr(B, res)
            z, nk = chebyshev_normal(lambda v: Nmat.T @ (B.T @ (B @ (Nmat @ v))), Nmat.T @ g,
                                     sL, sU, refine_tol)
            xf = xf + Nmat @ z
            steps.append(nk)
        x = xf
    else:
        info["M"] = Mmat
        for _ in range(refine):
            res = dd_residual(B, b, sol)
            d_, it = chebyshev(matvec, rmatvec, Mmat.T @ res, dim, sL, sU, refine_tol)
            sol = sol + d_
            steps.append(it["iterations"])
        x = sol[:n] / lam if lam > 0 else sol
    info["refine_steps"] = steps
    return x, info


# --------------------------------------------------------------------------- #
# Acceptance metrics                                                           #
# --------------------------------------------------------------------------- #
def rel_err(x: np.ndarray, xstar: np.ndarray) -> float:
    den = float(np.linalg.norm(xstar))
    return float(np.linalg.norm(np.asarray(x) - xstar)) / (den if den > 0 else 1.0)


def two_norm_estimate(A, iters: int = 30, seed: int = 1) -> float:
    """||A||_2 by power iteration on A^T A (dense or sparse A)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(A.shape[1])
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        w = np.asarray(A.T @ (A @ v)).ravel()
        est = math.sqrt(float(np.linalg.norm(w)))
        v = w / np.linalg.norm(w)
    return est


def normal_eq_residual(A, b: np.ndarray, x: np.ndarray, anorm: Optional[float] = None) -> float:
    """||A^T r|| / (||A||_2 ||r||), r = b - A x (FP64; A dense or sparse)."""
    r = b - np.asarray(A @ x).ravel()
    atr = np.asarray(A.T @ r).ravel()
    if anorm is None:
        anorm = two_norm_estimate(A)
    rn = float(np.linalg.norm(r))
    if rn == 0.0:
        return 0.0
    return float(np.linalg.norm(atr)) / (anorm * rn)
