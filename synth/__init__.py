"""Seeded synthetic least-squares inputs shaped like the paper's workloads.

This module holds input generation only (no sketching, no solving): both the
oracle-based tests and the CUDA path are fed from it.  The benchmark setup of the
paper (Sec. 3.1) uses ill-conditioned Gaussian-based matrices; no dataset is
involved, so every input here is synthetic and reproducible from its seed.

Recipes:

* ``gaussian_problem``: A iid N(0,1), x_true iid N(0,1), b = A x_true + noise * N(0,1).
* ``ill_conditioned_problem``: A = G diag(sigma) Q with G iid N(0,1) (m x n), Q a
  Haar-random orthogonal n x n (QR of a Gaussian with the signs of diag(R) moved
  into Q, Mezzadri 2007), sigma_j = kappa^(-j/(n-1)) (log-spaced from 1 to
  1/kappa), x_true iid N(0,1), b = A x_true + noise * N(0,1).
* ``paper_problem``: the benchmark setup the paper follows (Epperly et al.
  2024): A = U diag(sigma) V^T with U (m x n) and V (n x n) Haar-random
  orthonormal, sigma_j = kappa^(-j/(n-1)); x* = w / ||w|| for Gaussian w;
  r* = beta * P z / ||P z|| with z Gaussian and P = I - U U^T, so r* is
  orthogonal to range(A); b = A x* + r*.  Then x* is the exact least-squares
  solution and ||b - A x*|| = beta by construction.  FP64.
* ``csr_problem``: per row a Binomial(n, density) count of uniformly random,
  distinct column positions with N(0,1) values, plus ``n_dense`` seeded rows that
  are fully dense and scaled by ``dense_scale`` (high-leverage rows);
  b = A x_true + noise * N(0,1).
* ``batched_shapes`` / ``served_requests``: the shape mixes of the batched and
  served workloads.

Matrices are produced in FP32 (or FP64 when asked) in chunks of rows, and b is
computed in FP64 from the stored matrix, then stored in the matrix dtype.
"""
import numpy as np

CHUNK = 1 << 16


def _rng(seed):
    return np.random.default_rng(int(seed))


def haar_orthogonal(n, rng):
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def log_spaced_sigma(n, kappa):
    if n == 1:
        return np.ones(1)
    return kappa ** (-np.arange(n) / (n - 1.0))


def _finish(A, x_true, noise, rng, dtype):
    m = A.shape[0]
    b = np.empty(m, dtype=np.float64)
    for r0 in range(0, m, CHUNK):
        r1 = min(m, r0 + CHUNK)
        b[r0:r1] = A[r0:r1].astype(np.float64) @ x_true
    b += noise * rng.standard_normal(m)
    return b.astype(dtype)


def gaussian_problem(m, n, seed, noise=1e-3, dtype=np.float64):
    """Dense iid N(0,1) matrix; returns (A, b, x_true)."""
    rng = _rng(seed)
    A = rng.standard_normal((m, n)).astype(dtype)
    x_true = rng.standard_normal(n)
    return A, _finish(A, x_true, noise, rng, dtype), x_true


def ill_conditioned_problem(m, n, seed, kappa=1e6, noise=1e-4, dtype=np.float32):
    """A = G diag(sigma) Q with condition number about kappa; returns (A, b, x_true)."""
    rng = _rng(seed)
    Q = haar_orthogonal(n, rng)
    Mx = log_spaced_sigma(n, kappa)[:, None] * Q
    A = np.empty((m, n), dtype=dtype)
    for r0 in range(0, m, CHUNK):
        r1 = min(m, r0 + CHUNK)
        G = rng.standard_normal((r1 - r0, n))
        A[r0:r1] = (G @ Mx).astype(dtype)
    x_true = rng.standard_normal(n)
    return A, _finish(A, x_true, noise, rng, dtype), x_true


def paper_problem(m, n, seed, kappa=1e10, beta=1e-10):
    """Ill-conditioned problem with a known solution; returns (A, b, x_star)."""
    rng = _rng(seed)
    U = haar_orthogonal_columns(m, n, rng)
    V = haar_orthogonal(n, rng)
    sigma = log_spaced_sigma(n, kappa)
    A = (U * sigma[None, :]) @ V.T
    w = rng.standard_normal(n)
    x_star = w / np.linalg.norm(w)
    z = rng.standard_normal(m)
    z -= U @ (U.T @ z)
    z -= U @ (U.T @ z)                  # twice: orthogonal to range(U) to rounding
    r_star = beta * z / np.linalg.norm(z)
    b = A @ x_star + r_star
    return A, b, x_star


def haar_orthogonal_columns(m, n, rng):
    """m x n matrix with orthonormal columns, Haar-distributed (QR of an m x n
    Gaussian with the signs of diag(R) moved into Q)."""
    Z = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


class CSR:
    """Plain CSR container: rowptr (int64, m+1), col (int32), val (float32)."""

    def __init__(self, m, n, rowptr, col, val):
        self.m, self.n = int(m), int(n)
        self.rowptr, self.col, self.val = rowptr, col, val

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def matvec(self, x):
        """A x in FP64 (input generation helper)."""
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        out = np.zeros(self.m)
        np.add.at(out, rows, self.val.astype(np.float64) * x[self.col])
        return out

    def to_dense(self):
        D = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        D[rows, self.col] = self.val
        return D


def csr_problem(m, n, seed, density=0.01, n_dense=64, dense_scale=100.0, noise=1e-3):
    """Sparse CSR matrix with uniformly random column positions; returns (csr, b, x_true)."""
    rng = _rng(seed)
    counts = rng.binomial(n, density, size=m).astype(np.int64)
    dense_rows = np.sort(rng.choice(m, size=min(n_dense, m), replace=False)) if n_dense else np.zeros(0, np.int64)
    counts[dense_rows] = 0
    rows = np.repeat(np.arange(m, dtype=np.int64), counts)
    cols = rng.integers(0, n, size=rows.size, dtype=np.int64)
    # distinct positions inside a row: drop repeated (row, col) pairs
    key = np.unique(rows * n + cols)
    rows, cols = key // n, key % n
    if dense_rows.size:
        rows = np.concatenate([rows, np.repeat(dense_rows, n)])
        cols = np.concatenate([cols, np.tile(np.arange(n, dtype=np.int64), dense_rows.size)])
        order = np.lexsort((cols, rows))
        rows, cols = rows[order], cols[order]
    val = rng.standard_normal(rows.size).astype(np.float32)
    if dense_rows.size:
        is_dense = np.isin(rows, dense_rows)
        val[is_dense] *= np.float32(dense_scale)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    A = CSR(m, n, rowptr, cols.astype(np.int32), val)
    x_true = rng.standard_normal(n)
    b = (A.matvec(x_true) + noise * rng.standard_normal(m)).astype(np.float32)
    return A, b, x_true


def batched_shapes(nprob, seed, m_lo=4096, m_hi=65536, n_choices=(16, 32, 64, 128), d_factor=4):
    """(m, n, d) per problem: m uniform in [m_lo, m_hi], n uniform over n_choices, d = d_factor*n."""
    rng = _rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=nprob)
    ns = rng.choice(np.asarray(n_choices), size=nprob)
    return [(int(m), int(n), int(d_factor * n)) for m, n in zip(ms, ns)]


def served_requests(nreq, seed, rate_per_s, m_lo_log2=14, m_hi_log2=22,
                    n_choices=(32, 64, 128, 256, 512, 1024), dens_lo=0.005, dens_hi=0.05,
                    tols=(1e-3, 1e-10)):
    """Poisson arrivals (exponential gaps at rate_per_s) with shapes: m log-uniform
    in [2^m_lo_log2, 2^m_hi_log2], n uniform over n_choices, half dense and half CSR
    (density uniform in [dens_lo, dens_hi]), tolerance chosen uniformly from tols."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=nreq)
    t = np.cumsum(gaps)
    ms = np.exp2(rng.uniform(m_lo_log2, m_hi_log2, size=nreq)).astype(np.int64)
    ns = rng.choice(np.asarray(n_choices), size=nreq)
    sparse = rng.random(nreq) < 0.5
    dens = rng.uniform(dens_lo, dens_hi, size=nreq)
    tol = rng.choice(np.asarray(tols), size=nreq)
    return [dict(t=float(t[i]), m=int(ms[i]), n=int(ns[i]), sparse=bool(sparse[i]),
                 density=float(dens[i]), tol=float(tol[i]), seed=int(seed) * 100003 + i)
            for i in range(nreq)]
