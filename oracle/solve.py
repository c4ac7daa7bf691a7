"""Solvers of the oracle, FP64.  TEST INFRASTRUCTURE ONLY.

* Householder QR and back substitution: standard solvers for the reduced
  problem min ||SA x^ - Sb||^2 (Sec. 1.2 step 3, Sec. 1.3).  Written out
  column by column: no blocking, no pivoting.
* Sketch-and-solve: QR of the augmented matrix [SA | Sb] (d x (n+1)).  Its R has
  R[:n, :n] = R, R[:n, n] = z = (Q^T Sb)[:n] and |R[n, n]| = ||SA x^ - Sb||.
* Exact least squares x* (the comparison point of the paper's forward- and
  residual-error figures, Sec. 3.2): the same QR applied to the full [A | b].
* LSQR (Paige & Saunders, ACM TOMS 8(1), 1982) on the right-preconditioned
  operator A R^{-1}: the sketch-and-precondition solver SAP-SAS the paper names in
  Sec. 2.1 (after Meier et al. 2023), started from the sketch-and-solve answer.
* eta(x) = ||A^T (b - A x)|| / (||A||_F ||b - A x||): the reading used for the
  unspecified "relative residual" (the Paige-Saunders normal-equation backward
  error measure; 0 exactly at x*).
"""
import numpy as np

U64 = np.finfo(np.float64).eps / 2


class RankDeficient(Exception):
    pass


def householder_qr(M):
    """Householder QR of a (p x q) matrix, p >= q.  Returns (R, V, tau): R upper
    triangular q x q, and the reflectors I - tau_j v_j v_j^T (v_j[j] = 1) with
    Q^T M = [R; 0].  Sign convention: R[j, j] = -sign(x_0) ||x|| (x_0 = 0 counts as
    positive), so no cancellation forming v."""
    W = np.array(M, dtype=np.float64, copy=True)
    p, q = W.shape
    assert p >= q
    V = np.zeros((p, q))
    tau = np.zeros(q)
    for j in range(q):
        x = W[j:, j]
        normx = np.sqrt(np.dot(x, x))
        if normx == 0.0:
            V[j, j] = 1.0
            continue
        alpha = -normx if x[0] >= 0 else normx
        v = x.copy()
        v[0] -= alpha
        v0 = v[0]
        v /= v0                                    # v[0] = 1
        t = -v0 / alpha                            # tau = 2 / (v^T v) for this scaling
        V[j:, j] = v
        tau[j] = t
        # apply I - t v v^T to the remaining columns
        w = v @ W[j:, j:]
        W[j:, j:] -= t * np.outer(v, w)
        W[j + 1:, j] = 0.0
        W[j, j] = alpha
    return np.triu(W[:q, :q]), V, tau


def apply_qt(V, tau, y):
    """Q^T y using the stored reflectors (y of length p)."""
    y = np.array(y, dtype=np.float64, copy=True)
    for j in range(V.shape[1]):
        v = V[j:, j]
        y[j:] -= tau[j] * v * np.dot(v, y[j:])
    return y


def back_solve(R, z):
    """x with R x = z, R upper triangular, by back substitution."""
    n = R.shape[0]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (z[i] - np.dot(R[i, i + 1:], x[i + 1:])) / R[i, i]
    return x


def forward_solve_transposed(R, z):
    """x with R^T x = z, R upper triangular (R^T lower), by forward substitution."""
    n = R.shape[0]
    x = np.zeros(n)
    for i in range(n):
        x[i] = (z[i] - np.dot(R[:i, i], x[:i])) / R[i, i]
    return x


def is_rank_deficient(R):
    """Reading of rank deficiency: |R_jj| <= n * u64 * max_i |R_ii|."""
    dg = np.abs(np.diag(R))
    return bool(np.any(dg <= R.shape[0] * U64 * dg.max())) if dg.size else True


def qr_solve_augmented(M, rhs):
    """Least-squares solve of min ||M x - rhs|| through the QR of [M | rhs].
    Returns (x, R, residual_norm) with R the n x n triangular factor of M."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[1]
    Raug, _, _ = householder_qr(np.column_stack([M, np.asarray(rhs, dtype=np.float64)]))
    R = Raug[:n, :n]
    if is_rank_deficient(R):
        raise RankDeficient()
    z = Raug[:n, n]
    return back_solve(R, z), R, abs(Raug[n, n])


def sketch_and_solve(SA, Sb):
    """x^ = argmin ||SA x - Sb|| (Sec. 1.3), with R of SA and ||SA x^ - Sb||."""
    return qr_solve_augmented(SA, Sb)


def exact_lstsq(A, b):
    """x* = argmin ||A x - b|| by Householder QR of [A | b] (FP64)."""
    x, _, rn = qr_solve_augmented(A, b)
    return x, rn


def eta(A, b, x):
    """||A^T r|| / (||A||_F ||r||), r = b - A x, all in FP64."""
    A = np.asarray(A, dtype=np.float64)
    r = np.asarray(b, dtype=np.float64) - A @ x
    nr = np.linalg.norm(r)
    if nr == 0.0:
        return 0.0
    return np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * nr)


def lsqr_preconditioned(A, b, R, x0, tol=1e-14, max_iter=1000):
    """LSQR on min ||(A R^{-1}) z - r0||, r0 = b - A x0; returns x = x0 + R^{-1} z,
    the iteration count and the estimate of ||(AR^-1)^T r|| / (||AR^-1||_F ||r||).

    Steps (Paige & Saunders 1982, Golub-Kahan bidiagonalisation with the QR
    update of the bidiagonal):  beta u = r0;  alpha v = M^T u;  w = v;
    phibar = beta;  rhobar = alpha;  then per iteration
      beta u = M v - alpha u;  alpha v = M^T u - beta v;
      rho = hypot(rhobar, beta);  c = rhobar/rho;  s = beta/rho;
      theta = s alpha;  rhobar = -c alpha;  phi = c phibar;  phibar = s phibar;
      z += (phi/rho) w;  w = v - (theta/rho) w;
    with stopping on the normal-equation estimate
      ||M^T r|| / (||M||_F ||r||) = (phibar alpha |c|) / (anorm phibar).
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]

    def M(v):
        return A @ back_solve(R, v)

    def Mt(u):
        return forward_solve_transposed(R, A.T @ u)

    r0 = np.asarray(b, dtype=np.float64) - A @ x0
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return np.array(x0, dtype=np.float64), 0, 0.0
    u = r0 / beta
    v = Mt(u)
    alpha = np.linalg.norm(v)
    if alpha == 0.0:
        return np.array(x0, dtype=np.float64), 0, 0.0
    v /= alpha
    w = v.copy()
    z = np.zeros(n)
    phibar, rhobar = beta, alpha
    anorm2 = alpha * alpha
    est = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        u = M(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0:
            u /= beta
        anorm2 += beta * beta
        v = Mt(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0:
            v /= alpha
        anorm2 += alpha * alpha
        rho = np.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        z += (phi / rho) * w
        w = v - (theta / rho) * w
        est = abs(alpha * c) / np.sqrt(anorm2)    # ||M^T r|| / (||M||_F ||r||)
        if est <= tol or alpha == 0.0:
            break
    return np.asarray(x0, dtype=np.float64) + back_solve(R, z), it, est


def sketch_and_precondition(A, b, SA, Sb, tol=1e-14, max_iter=1000):
    """SAP-SAS: sketch-and-solve start x^ from QR(SA), then LSQR on A R^{-1}.
    Its fixed point is x* (pinned through exact_lstsq)."""
    xhat, R, _ = sketch_and_solve(SA, Sb)
    x, it, est = lsqr_preconditioned(A, b, R, xhat, tol=tol, max_iter=max_iter)
    return x, it, est, xhat


def apply_inverse_r(A, R):
    """Y = A R^{-1} formed explicitly (the "apply" of sketch-and-apply), column
    by column from Y R = A: Y[:, j] = (A[:, j] - Y[:, :j] R[:j, j]) / R[j, j]."""
    A = np.asarray(A, dtype=np.float64)
    n = R.shape[0]
    Y = np.zeros_like(A)
    for j in range(n):
        Y[:, j] = (A[:, j] - Y[:, :j] @ R[:j, j]) / R[j, j]
    return Y


def sketch_and_apply(A, b, SA, Sb, tol=1e-14, max_iter=1000):
    """SAA-SAS (named in Sec. 2.1 beside SAP-SAS; after Meier, Nakatsukasa,
    Townsend & Webb 2023): R from the QR of SA, Y = A R^{-1} formed explicitly,
    LSQR on min ||Y z - b|| started at z0 = R x^ (x^ the sketch-and-solve
    solution), and x = R^{-1} z.  Returns x, the iteration count, LSQR's
    estimate of ||Y^T r|| / (||Y||_F ||r||) and x^."""
    xhat, R, _ = sketch_and_solve(SA, Sb)
    n = R.shape[0]
    Y = apply_inverse_r(A, R)
    z, it, est = lsqr_preconditioned(Y, b, np.eye(n), R @ xhat, tol=tol, max_iter=max_iter)
    return back_solve(R, z), it, est, xhat
