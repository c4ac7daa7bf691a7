"""Pins of the oracle's solvers: LAPACK/SciPy routines, consistent systems,
identity/permutation sketches, brute-force normal equations, closed forms."""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.sparse.linalg import lsqr as scipy_lsqr

from oracle import sketch as S
from oracle import solve as L
from synth import gaussian_problem, ill_conditioned_problem


def _q_from(V, tau):
    p = V.shape[0]
    Q = np.eye(p)
    for j in reversed(range(V.shape[1])):      # Q = H_0 H_1 ... H_{q-1}
        v = V[j:, j]
        Q[j:, :] -= tau[j] * np.outer(v, v @ Q[j:, :])
    return Q


@pytest.mark.parametrize("shape", [(1, 1), (5, 5), (40, 7), (257, 64)])
def test_householder_qr_factorisation(shape):
    rng = np.random.default_rng(shape[0])
    M = rng.standard_normal(shape)
    R, V, tau = L.householder_qr(M)
    Q = _q_from(V, tau)
    q = shape[1]
    assert np.allclose(Q.T @ Q, np.eye(shape[0]), atol=1e-13)
    assert np.allclose(Q[:, :q] @ R, M, atol=1e-13)
    assert np.array_equal(R, np.triu(R))
    Rl = np.linalg.qr(M, mode="r")             # LAPACK geqrf
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-12)
    y = rng.standard_normal(shape[0])
    assert np.allclose(L.apply_qt(V, tau, y), Q.T @ y, atol=1e-12)


def test_triangular_solves_match_scipy():
    rng = np.random.default_rng(1)
    R = np.triu(rng.standard_normal((30, 30))) + 5 * np.eye(30)
    z = rng.standard_normal(30)
    assert np.allclose(L.back_solve(R, z), sla.solve_triangular(R, z), rtol=1e-12)
    assert np.allclose(L.forward_solve_transposed(R, z), sla.solve_triangular(R, z, trans="T"), rtol=1e-12)


def test_exact_lstsq_matches_lapack():
    A, b, _ = ill_conditioned_problem(2000, 30, seed=3, kappa=1e4, noise=1e-3, dtype=np.float64)
    x, rn = L.exact_lstsq(A, b)
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e4 * 1e-14
    assert np.isclose(rn, np.linalg.norm(A @ xr - b), rtol=1e-10)


def test_consistent_system_recovers_x_true():
    # paper config 1 shape: 4096 x 64 FP64 N(0,1), CountSketch d = 256, seed 0
    A, _, x_true = gaussian_problem(4096, 64, seed=1001)
    b = A @ x_true
    SA, Sb = S.countsketch_apply(A, 256, 0), S.countsketch_apply(b, 256, 0)
    x, _, rn = L.sketch_and_solve(SA, Sb)
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) < 1e-13
    assert rn < 1e-10


def test_identity_and_permutation_sketch_reduce_to_plain_lstsq():
    A, b, _ = gaussian_problem(200, 6, seed=2, noise=1.0)
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    x, _, _ = L.sketch_and_solve(A, b)
    assert np.allclose(x, xr, rtol=1e-12, atol=1e-13)
    perm = np.random.default_rng(0).permutation(200)
    x2, _, _ = L.sketch_and_solve(A[perm], b[perm])
    assert np.allclose(x2, xr, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("kind", S.KINDS)
def test_sketch_and_solve_brute_force_normal_equations(kind):
    A, b, _ = gaussian_problem(120, 5, seed=7, noise=0.5)
    d = 32
    SA, Sb = S.sketch_apply(kind, A, d, 3, bf16_operand=False), S.sketch_apply(kind, b, d, 3, bf16_operand=False)
    x, _, rn = L.sketch_and_solve(SA, Sb)
    xn = np.linalg.solve(SA.T @ SA, SA.T @ Sb)
    assert np.allclose(x, xn, rtol=1e-9, atol=1e-12)
    assert np.isclose(rn, np.linalg.norm(SA @ x - Sb), rtol=1e-10)


@pytest.mark.parametrize("kind", S.KINDS)
def test_residual_ratio_bound_config1(kind):
    A, b, _ = gaussian_problem(4096, 64, seed=1001)
    x_star, rn = L.exact_lstsq(A, b)
    SA, Sb = S.sketch_apply(kind, A, 256, 0, bf16_operand=False), S.sketch_apply(kind, b, 256, 0, bf16_operand=False)
    x, _, _ = L.sketch_and_solve(SA, Sb)
    ratio = np.linalg.norm(A @ x - b) / rn
    assert 1.0 <= ratio <= 2.0


def test_rank_deficient_detected():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((50, 4))
    A[:, 3] = A[:, 0] + A[:, 1]
    with pytest.raises(L.RankDeficient):
        L.sketch_and_solve(A, rng.standard_normal(50))


def test_eta_zero_at_solution_and_positive_elsewhere():
    A, b, _ = gaussian_problem(500, 10, seed=4, noise=0.1)
    x, _ = L.exact_lstsq(A, b)
    assert L.eta(A, b, x) < 1e-14
    assert L.eta(A, b, x + 1e-3) > 1e-6


def test_eta_hand_computed_values():
    """eta = ||A^T r|| / (||A||_F ||r||) on a 3 x 2 problem worked by hand:
    A = [[3, 0], [0, 4], [0, 0]] has ||A||_F = 5; with b = (1, 1, 1):
    x = 0 gives r = b, A^T r = (3, 4): eta = 5 / (5 sqrt 3);
    x = (0, 1/4) gives r = (1, 0, 1), A^T r = (3, 0): eta = 3 / (5 sqrt 2);
    x = (1/3, 1/4) is x* (r = (0, 0, 1) is orthogonal to range(A)): eta = 0."""
    A = np.array([[3.0, 0.0], [0.0, 4.0], [0.0, 0.0]])
    b = np.ones(3)
    assert np.isclose(L.eta(A, b, np.zeros(2)), 1 / np.sqrt(3), rtol=1e-15)
    assert np.isclose(L.eta(A, b, np.array([0.0, 0.25])), 3 / (5 * np.sqrt(2)), rtol=1e-15)
    assert L.eta(A, b, np.array([1 / 3, 0.25])) < 1e-16


def test_eta_closed_form_scaled_orthonormal_columns():
    """A = c Q with Q^T Q = I (n columns), so ||A||_F = c sqrt(n).  With
    b = A x + p + Q w, p orthogonal to range(Q): r = p + Q w, A^T r = c w, so
    eta(x) = ||w|| / (sqrt(n) sqrt(||p||^2 + ||w||^2)), whatever c is.  Dividing
    by ||A||_2 instead of ||A||_F, or by ||r||^2, changes the value."""
    rng = np.random.default_rng(31)
    m, n = 60, 4
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    z = rng.standard_normal(m)
    p = z - Q @ (Q.T @ z)
    p *= 4.0 / np.linalg.norm(p)                     # ||p|| = 4
    w = np.array([1.0, 2.0, 2.0, 0.0])               # ||w|| = 3
    x = rng.standard_normal(n)
    for c in (1.0, 7.5, 1e-3):
        A = c * Q
        b = A @ x + p + Q @ w
        assert np.isclose(L.eta(A, b, x), 3.0 / (2.0 * 5.0), rtol=1e-12)   # 3 / (sqrt(4) * 5)


def test_eta_scale_invariance():
    """eta is a relative measure: scaling A and b together, or b and x
    together, leaves it unchanged (a squared norm anywhere would not)."""
    A, b, _ = gaussian_problem(300, 8, seed=32, noise=0.2)
    x = np.random.default_rng(33).standard_normal(8)
    e = L.eta(A, b, x)
    assert np.isclose(L.eta(9.0 * A, 9.0 * b, x), e, rtol=1e-12)
    assert np.isclose(L.eta(A, 0.01 * b, 0.01 * x), e, rtol=1e-12)


def test_eta_matches_scipy_lsqr_recurrence():
    """SciPy's LSQR carries ||A^T r_k|| (arnorm) and ||r_k|| (r1norm) of its
    iterate through its own recurrences; at that iterate they give the same
    eta as the oracle's direct computation."""
    A, b, _ = gaussian_problem(400, 10, seed=34, noise=0.5)
    fro = np.sqrt(np.sum(A * A))
    for k in (2, 4, 7):
        out = scipy_lsqr(A, b, atol=0, btol=0, iter_lim=k)
        xk, r1norm, arnorm = out[0], out[3], out[7]
        assert np.isclose(L.eta(A, b, xk), arnorm / (fro * r1norm), rtol=1e-8)


def test_lsqr_iterates_match_scipy_lsqr():
    # with R = I the iteration is plain LSQR: compare iterates after k steps
    A, b, _ = gaussian_problem(300, 12, seed=5, noise=0.3)
    for k in (1, 3, 6):
        x, it, _ = L.lsqr_preconditioned(A, b, np.eye(12), np.zeros(12), tol=0.0, max_iter=k)
        xs = scipy_lsqr(A, b, atol=0, btol=0, iter_lim=k)[0]
        assert it == k
        assert np.allclose(x, xs, rtol=1e-10, atol=1e-12)


def test_sap_fixed_point_is_exact_solution_ill_conditioned():
    A, b, _ = ill_conditioned_problem(3000, 20, seed=6, kappa=1e8, noise=1e-4, dtype=np.float64)
    x_star, _ = L.exact_lstsq(A, b)
    SA, Sb = S.countsketch_apply(A, 80, 1), S.countsketch_apply(b, 80, 1)
    x, it, est, xhat = L.sketch_and_precondition(A, b, SA, Sb, tol=1e-15, max_iter=200)
    assert np.linalg.norm(x - x_star) / np.linalg.norm(x_star) < 1e8 * 1e-14
    # eta at the FP64 rounding floor of forming r itself (that of LAPACK's answer)
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    assert L.eta(A, b, x) < 10 * L.eta(A, b, xr) + 1e-14
    # preconditioned LSQR needs far fewer iterations than plain LSQR here
    _, it_plain, _ = L.lsqr_preconditioned(A, b, np.eye(20), xhat, tol=1e-10, max_iter=200)
    assert it < it_plain


# ---------------------------------------------------------------- sketch-and-apply (SAA-SAS)

def test_apply_inverse_r_reconstructs_and_matches_triangular_solve():
    from scipy.linalg import solve_triangular
    A, _, _ = gaussian_problem(400, 9, seed=21)
    _, R, _ = L.sketch_and_solve(S.countsketch_apply(A, 40, 3), S.countsketch_apply(np.ones(400), 40, 3))
    Y = L.apply_inverse_r(A, R)
    assert np.allclose(Y @ R, A, rtol=0, atol=1e-12 * np.abs(A).max())
    # Y^T = R^{-T} A^T by the library's triangular solve
    assert np.allclose(Y, solve_triangular(R, A.T, trans="T").T, rtol=1e-12, atol=1e-13)


def test_saa_fixed_point_is_exact_solution_ill_conditioned():
    A, b, _ = ill_conditioned_problem(3000, 20, seed=22, kappa=1e8, noise=1e-4, dtype=np.float64)
    x_star, _ = L.exact_lstsq(A, b)
    SA, Sb = S.countsketch_apply(A, 80, 1), S.countsketch_apply(b, 80, 1)
    x, it, est, xhat = L.sketch_and_apply(A, b, SA, Sb, tol=1e-15, max_iter=200)
    assert np.linalg.norm(x - x_star) / np.linalg.norm(x_star) < 1e8 * 1e-14
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    assert L.eta(A, b, x) < 10 * L.eta(A, b, xr) + 1e-14


def test_saa_iterates_equal_sap_iterates():
    """LSQR on the explicit Y = A R^{-1} from z0 = R x^ and LSQR on the implicit
    A R^{-1} from x^ build the same Krylov iterates: mapped back, the k-th
    iterates agree (up to rounding at this moderate conditioning)."""
    A, b, _ = ill_conditioned_problem(2000, 15, seed=23, kappa=1e3, noise=1e-2, dtype=np.float64)
    SA, Sb = S.countsketch_apply(A, 60, 2), S.countsketch_apply(b, 60, 2)
    for k in (1, 2, 5):
        xa, ita, _, _ = L.sketch_and_apply(A, b, SA, Sb, tol=0.0, max_iter=k)
        xp, itp, _, _ = L.sketch_and_precondition(A, b, SA, Sb, tol=0.0, max_iter=k)
        assert ita == itp == k
        assert np.linalg.norm(xa - xp) / np.linalg.norm(xp) < 1e-10


def test_saa_preconditioned_matrix_is_well_conditioned():
    """With d = 4n the sketch keeps the singular values of A R^{-1} near 1
    (subspace embedding): kappa(Y) stays small whatever kappa(A) is."""
    A, _, _ = ill_conditioned_problem(4000, 16, seed=24, kappa=1e8, noise=0.0, dtype=np.float64)
    _, R, _ = L.sketch_and_solve(S.countsketch_apply(A, 64, 5), S.countsketch_apply(np.ones(4000), 64, 5))
    assert np.linalg.cond(L.apply_inverse_r(A, R)) < 6.0
