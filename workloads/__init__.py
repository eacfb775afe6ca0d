"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds inputs (A, b and the factors they were built from).  It
holds none of LSRN's arithmetic: no sketch, no SVD of the sketch, no LSQR or
Chebyshev step, and not the Philox/Box-Muller generator of the sketching
matrix.  Its random numbers come from numpy's PCG64 streams, which are the same
on every platform.  Both the oracle and the CUDA path consume the bytes made
here, so a test always compares the two on identical inputs.

Workload families (the paper's experiments use random matrices with a prescribed
condition number and rank, section 6.2 and 6.4, and sprandn-like sparse
matrices, section 6.5):

* ``dense_haar``        -- A = U diag(sigma) V^T with Haar-distributed U, V
                           (QR of a Gaussian matrix, signs fixed by diag(R) > 0),
                           sigma log-spaced from 1 to 1/cond on the first `rank`
                           entries, zeros after; b = A x0 + noise * N(0, 1).
* ``dense_householder`` -- same spectrum, but U = H_1..H_k [I_r; 0] and
                           V = H'_1..H'_k [I_r; 0] from k seeded Householder
                           reflectors, so that a 10^6 x 2000 matrix can be built
                           in one pass (compact WY form, rank-k update).
* ``csr_uniform_rows``  -- CSR with a fixed number of distinct, uniformly drawn,
                           sorted columns per row and N(0, 1) values.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np


def log_spaced_sigma(rank: int, cond: float) -> np.ndarray:
    """sigma_i = cond^(-(i-1)/(rank-1)), i = 1..rank (1 -> 1/cond)."""
    if rank <= 0:
        return np.zeros(0)
    if rank == 1:
        return np.ones(1)
    return np.power(10.0, -np.log10(cond) * np.arange(rank) / (rank - 1))


@dataclasses.dataclass
class DenseProblem:
    A: object                       # numpy (m, n) float64 C-contiguous, or a torch tensor
    b: object                       # (m,)
    x0: np.ndarray                  # (n,)
    sigma: np.ndarray               # (rank,) planted singular values
    apply_Ut: Callable[[np.ndarray], np.ndarray]   # b (m,) -> U^T b (rank,)
    apply_V: Callable[[np.ndarray], np.ndarray]    # c (rank,) -> V c (n,)
    meta: dict
    apply_U: Optional[Callable[[np.ndarray], np.ndarray]] = None    # c (rank,) -> U c (m,)
    apply_Vt: Optional[Callable[[np.ndarray], np.ndarray]] = None   # v (n,) -> V^T v (rank,)


def _haar(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((n, k)))
    return q * np.sign(np.diag(r))


def dense_haar(m: int, n: int, rank: int, cond: float, noise: float, seed: int) -> DenseProblem:
    """Dense A = U diag(sigma) V^T with Haar factors (the 2000 x 100 recipe)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    U = _haar(rng, m, rank)
    V = _haar(rng, n, rank)
    sigma = log_spaced_sigma(rank, cond)
    A = np.ascontiguousarray((U * sigma) @ V.T)
    x0 = rng.standard_normal(n)
    b = A @ x0 + noise * rng.standard_normal(m)
    return DenseProblem(A=A, b=b, x0=x0, sigma=sigma,
                        apply_Ut=lambda v: U.T @ v, apply_V=lambda c: V @ c,
                        meta=dict(kind="haar", m=m, n=n, rank=rank, cond=cond,
                                  noise=noise, seed=seed, U=U, V=V))


class _Reflectors:
    """Q = H_1 ... H_k = I - Y T Y^T with H_i = I - tau_i y_i y_i^T (compact WY)."""

    def __init__(self, Y: np.ndarray):
        self.Y = Y
        k = Y.shape[1]
        tau = 2.0 / np.einsum("ij,ij->j", Y, Y)
        T = np.zeros((k, k))
        gram = Y.T @ Y
        for i in range(k):
            T[i, i] = tau[i]
            if i:
                T[:i, i] = -tau[i] * (T[:i, :i] @ gram[:i, i])
        self.T = T

    def apply(self, X: np.ndarray) -> np.ndarray:     # Q X
        return X - self.Y @ (self.T @ (self.Y.T @ X))

    def apply_t(self, X: np.ndarray) -> np.ndarray:   # Q^T X
        return X - self.Y @ (self.T.T @ (self.Y.T @ X))


def dense_householder(m: int, n: int, rank: int, cond: float, noise: float, seed: int,
                      n_reflectors: int = 8, device: Optional[str] = None,
                      row_block: int = 65536, rows: Optional[tuple] = None) -> DenseProblem:
    """Dense A = U diag(sigma) V^T with U, V products of seeded Householder reflectors.

    A = Q [W; 0] with W = diag(sigma) V^T (rank x n) and Q = I - Y T Y^T, so
    A = [W; 0] - Y (T Y[:rank]^T W): a rank-k update written row block by row
    block.  With ``device`` set (a torch device string) A and b are built there
    with torch, otherwise with numpy on the host.  With ``rows = (r0, r1)``
    (device path) only rows r0 .. r1 - 1 of A and b are built -- one shard of a
    row-partitioned problem; the factors (apply_Ut, ...) stay those of the
    whole matrix.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    k = n_reflectors
    QU = _Reflectors(rng.standard_normal((m, k)))
    QV = _Reflectors(rng.standard_normal((n, k)))
    sigma = log_spaced_sigma(rank, cond)
    eye = np.zeros((n, rank))
    eye[:rank, :rank] = np.eye(rank)
    V = QV.apply(eye)                                   # n x rank
    W = sigma[:, None] * V.T                            # rank x n
    Z = QU.T @ (QU.Y[:rank].T @ W)                      # k x n
    x0 = rng.standard_normal(n)
    e = rng.standard_normal(m)
    if device is None:
        A = np.empty((m, n))
        for r0 in range(0, m, row_block):
            r1 = min(m, r0 + row_block)
            blk = -(QU.Y[r0:r1] @ Z)
            if r0 < rank:
                t = min(r1, rank)
                blk[: t - r0] += W[r0:t]
            A[r0:r1] = blk
        b = A @ x0 + noise * e
    else:
        import torch
        dev = torch.device(device)
        lo, hi = rows if rows is not None else (0, m)
        A = torch.empty((hi - lo, n), dtype=torch.float64, device=dev)
        Zt = torch.from_numpy(Z).to(dev)
        Wt = torch.from_numpy(W).to(dev)
        Yt = torch.from_numpy(QU.Y).to(dev)
        for r0 in range(lo, hi, row_block):
            r1 = min(hi, r0 + row_block)
            blk = -(Yt[r0:r1] @ Zt)
            if r0 < rank:
                t = min(r1, rank)
                blk[: t - r0] += Wt[r0:t]
            A[r0 - lo:r1 - lo] = blk
        b = A @ torch.from_numpy(x0).to(dev) + noise * torch.from_numpy(e[lo:hi]).to(dev)

    def apply_Ut(v: np.ndarray) -> np.ndarray:
        return QU.apply_t(np.asarray(v, dtype=np.float64).reshape(m, 1))[:rank, 0]

    def apply_V(c: np.ndarray) -> np.ndarray:
        return V @ np.asarray(c, dtype=np.float64)

    def apply_U(c: np.ndarray) -> np.ndarray:
        z = np.zeros((m, 1))
        z[:rank, 0] = np.asarray(c, dtype=np.float64)
        return QU.apply(z)[:, 0]

    def apply_Vt(v: np.ndarray) -> np.ndarray:
        return V.T @ np.asarray(v, dtype=np.float64)

    return DenseProblem(A=A, b=b, x0=x0, sigma=sigma, apply_Ut=apply_Ut, apply_V=apply_V,
                        apply_U=apply_U, apply_Vt=apply_Vt,
                        meta=dict(kind="householder", m=m, n=n, rank=rank, cond=cond,
                                  noise=noise, seed=seed, n_reflectors=k, V=V))


@dataclasses.dataclass
class CsrMatrix:
    m: int
    n: int
    row_ptr: np.ndarray      # int64 (m + 1,)
    col_idx: np.ndarray      # int32 (nnz,)
    values: np.ndarray       # float64 or float32 (nnz,)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        D = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        D[rows, self.col_idx] = self.values.astype(np.float64)
        return D


def csr_uniform_rows(m: int, n: int, nnz_per_row: int, seed: int,
                     dtype=np.float64) -> CsrMatrix:
    """Each row: `nnz_per_row` distinct columns drawn uniformly, sorted; N(0,1) values.

    With dtype float32 the values are the float64 draws rounded to float32.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    k = min(nnz_per_row, n)
    cols = np.empty((m, k), dtype=np.int32)
    for i in range(m):
        cols[i] = np.sort(rng.choice(n, size=k, replace=False, shuffle=False))
    vals = rng.standard_normal(m * k).astype(dtype)
    row_ptr = np.arange(0, (m + 1) * k, k, dtype=np.int64)
    return CsrMatrix(m=m, n=n, row_ptr=row_ptr, col_idx=cols.reshape(-1), values=vals)


def csr_random_density(m: int, n: int, density: float, seed: int,
                       dtype=np.float64) -> CsrMatrix:
    """sprandn-like CSR: each entry present independently with probability `density`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.binomial(n, density, size=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(counts)
    cols = np.empty(int(row_ptr[-1]), dtype=np.int32)
    for i in range(m):
        c = counts[i]
        if c:
            cols[row_ptr[i]:row_ptr[i + 1]] = np.sort(rng.choice(n, size=c, replace=False,
                                                                 shuffle=False))
    vals = rng.standard_normal(int(row_ptr[-1])).astype(dtype)
    return CsrMatrix(m=m, n=n, row_ptr=row_ptr, col_idx=cols, values=vals)


def gaussian_vector(n: int, seed: int) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


# Named recipes: the small parity case and the full-size benchmark case.
def c1_problem(seed: int = 0) -> DenseProblem:
    """2000 x 100, rank 80, sigma 1 -> 1e-6, Haar factors, noise 1e-3."""
    return dense_haar(2000, 100, 80, 1e6, 1e-3, seed)


def c2_problem(seed: int = 0, device: Optional[str] = None, m: int = 1_000_000,
               n: int = 2000, rank: int = 1800, rows: Optional[tuple] = None) -> DenseProblem:
    """10^6 x 2000, rank 1800, sigma 1 -> 1e-6, 8 Householder reflectors, noise 1e-4."""
    return dense_householder(m, n, rank, 1e6, 1e-4, seed, device=device, rows=rows)


def c3_problem(seed: int = 0, m: int = 10_000, n: int = 1_000_000, nnz_per_row: int = 2000,
               dtype=np.float64):
    """10^4 x 10^6 CSR, 2000 uniform columns per row, N(0,1) values; b ~ N(0,1)."""
    A = csr_uniform_rows(m, n, nnz_per_row, seed, dtype)
    b = gaussian_vector(m, seed + 7919)
    return A, b



def serving_mix(count: int, seed: int = 7, device: Optional[str] = None,
                m_range=(5_000, 200_000), n_range=(32, 512), tall_frac: float = 0.7,
                log10_cond=(2.0, 6.0)):
    """Request sizes and problems of the batched / serving mix: m log-uniform in
    m_range, n log-uniform in n_range, a fraction `tall_frac` stored m x n (the rest
    as its n x m transpose), rank u * min(m, n) with u ~ U[0.8, 1], condition number
    10^U[log10_cond], Householder-product factors, noise 1e-4.
    Returns a list of (DenseProblem, tall) with the problem generated tall
    (the fat request is its transpose)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        tall = bool(rng.random() < tall_frac)
        rank = max(1, int(math.ceil(rng.uniform(0.8, 1.0) * min(m, n))))
        cond = 10.0 ** rng.uniform(*log10_cond)
        P = dense_householder(m, n, rank, cond, 1e-4, seed * 100_003 + k, device=device)
        out.append((P, tall))
    return out


def csr_sprandn(m: int, n: int, density: float, seed: int, dtype=np.float64) -> CsrMatrix:
    """sprandn-like CSR built in bulk: row i holds Binomial(n, density) columns
    drawn uniformly (repeats within a row merged), values N(0,1), columns sorted."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.binomial(n, density, size=m)
    rows = np.repeat(np.arange(m, dtype=np.int64), counts)
    cols = rng.integers(0, n, size=rows.size, dtype=np.int64)
    key = np.unique(rows * n + cols)
    rows, cols = key // n, key % n
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(rows, minlength=m))
    vals = rng.standard_normal(key.size).astype(dtype)
    return CsrMatrix(m=m, n=n, row_ptr=row_ptr, col_idx=cols.astype(np.int32), values=vals)


def serving_requests(count: int, seed: int = 7, device: Optional[str] = None,
                     sparse_frac: float = 0.2, lambdas=(0.0, 1e-4, 1e-2)):
    """The serving mix: a fraction 1 - sparse_frac of dense problems drawn as in
    serving_mix (batched configuration, condition 1e2-1e6), the rest sparse:
    sprandn-like CSR with density 1e-3, short side log-uniform [32, 2000], long
    side log-uniform [1e5, 2e6], half of them tall; lambda drawn uniformly from
    `lambdas`.  Returns dicts with kind ('dense' / 'csr'), lam, and for dense the
    problem P and its orientation (fat requests are P.A^T), for CSR the matrix."""
    rng = np.random.Generator(np.random.PCG64(seed + 77))
    dense = iter(serving_mix(count, seed=seed, device=device))
    out = []
    for k in range(count):
        lam = float(lambdas[int(rng.integers(0, len(lambdas)))])
        if rng.random() < sparse_frac:
            short = int(round(math.exp(rng.uniform(math.log(32), math.log(2000)))))
            long = int(round(math.exp(rng.uniform(math.log(1e5), math.log(2e6)))))
            tall = bool(rng.random() < 0.5)
            m, n = (long, short) if tall else (short, long)
            C = csr_sprandn(m, n, 1e-3, seed * 1_000_003 + k)
            b = rng.standard_normal(m)
            out.append(dict(kind="csr", lam=lam, csr=C, b=b, tall=tall))
            next(dense)
        else:
            P, tall = next(dense)
            out.append(dict(kind="dense", lam=lam, P=P, tall=tall))
    return out
