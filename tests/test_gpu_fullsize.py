"""The benchmark's full-size problem (2^20 x 256 FP32, A = G diag(sigma) Q with
kappa = 1e6, noise 1e-4; CountSketch d = 1024, sketch seed 1: the launch
configuration bench.py times), checked with what the oracle can compute at
this size: the normal-equation backward error eta(x) = ||A^T(b - Ax)|| /
(||A||_F ||b - Ax||) in FP64 over the whole matrix (Sec. 2.1, SAP-SAS to a
tolerance), and sampled output rows of the Gaussian and SRHT sketches from
their definitions (Sec. 1.2.1)."""
import numpy as np
import pytest

from gpu_util import ctx, dev, rel_fro
from oracle import sketch as OS
from oracle import solve as OL
from synth import ill_conditioned_problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

M, N, D = 1 << 20, 256, 1024


@pytest.fixture(scope="module")
def problem():
    A, b, _ = ill_conditioned_problem(M, N, seed=1002, kappa=1e6, noise=1e-4)
    return A, b


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_full_size_solve_reaches_tol(problem, tol):
    A, b = problem
    c = ctx()
    x, info = c.lstsq(dev(A), dev(b), D, seed=1, tol=tol, max_iter=400)
    assert info.status == 0, info.status
    eta = OL.eta(A.astype(np.float64), b.astype(np.float64), x.cpu().numpy())
    assert eta <= 1.5 * tol, (eta, info.eta)


@pytest.fixture(scope="module")
def x_star(problem):
    """x* of the full-size problem by the oracle's FP64 sketch-and-precondition
    (LSQR on A R^-1 to 1e-14; its fixed point is pinned to the Householder x* by
    the oracle's own tests), a few seconds instead of a full-size QR."""
    A, b = problem
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    SA, Sb = OS.countsketch_apply(A64, D, 1), OS.countsketch_apply(b64, D, 1)
    x, _, est, _ = OL.sketch_and_precondition(A64, b64, SA, Sb, tol=1e-14, max_iter=400)
    assert est <= 1e-13
    return x


def test_full_size_forward_error_at_fp64_floor(problem, x_star):
    """Run to the FP64-class floor, the solution agrees with x* to the FP64
    perturbation bound kappa * u64 (times a small constant), kappa = 1e6."""
    A, b = problem
    c = ctx()
    x, info = c.lstsq(dev(A), dev(b), D, seed=1, tol=1e-12, max_iter=400)
    err = np.linalg.norm(x.cpu().numpy() - x_star) / np.linalg.norm(x_star)
    print(f"forward error at the floor: {err:.3e} (status {info.status}, {info.iters} passes)")
    assert err <= 100 * 1e6 * 2.0 ** -53, err


def test_full_size_forward_error_follows_eta(problem, x_star):
    """At eta <= 1e-6 and 1e-10 the distance to x* is what the backward error
    allows: x - x* = -(A^T A)^{-1} A^T r(x) exactly, so ||x - x*|| <= ||A^T r|| /
    s_min(A)^2.  s_min(A) >= s_min(A R^-1) s_min(R) with R from the oracle's QR of
    an FP64 sketch; A R^-1 is well conditioned, so its Gram matrix gives its
    smallest singular value accurately in FP64."""
    A, b = problem
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    c = ctx()
    _, R, _ = OL.sketch_and_solve(OS.countsketch_apply(A64, D, 1), OS.countsketch_apply(b64, D, 1))
    from scipy.linalg import solve_triangular
    Y = solve_triangular(R, A64.T, trans="T").T            # A R^-1
    s_min = np.sqrt(np.linalg.eigvalsh(Y.T @ Y)[0]) * np.linalg.svd(R, compute_uv=False)[-1]
    del Y
    for tol in (1e-6, 1e-10):
        x, info = c.lstsq(dev(A), dev(b), D, seed=1, tol=tol, max_iter=400)
        xg = x.cpu().numpy()
        g = A64.T @ (b64 - A64 @ xg)
        err = np.linalg.norm(xg - x_star) / np.linalg.norm(x_star)
        bound = np.linalg.norm(g) / s_min ** 2 / np.linalg.norm(x_star)
        print(f"tol {tol:g}: forward error {err:.3e} (bound {bound:.3e})")
        assert info.status == 0
        assert err <= bound + 100 * 1e6 * 2.0 ** -53, (err, bound)


@pytest.mark.parametrize("terms", [1, 3])
def test_full_size_gaussian_sampled_rows(problem, terms):
    A, b = problem
    c = ctx()
    SA, Sb = c.sketch(dev(A), dev(b), D, kind="gaussian", seed=1, variant=str(terms))
    rows = [0, 7, 8, 31, 32, 500, 1023]
    ref = OS.gaussian_rows(A, D, 1, rows, terms=terms)
    refb = OS.gaussian_rows(b, D, 1, rows, terms=terms)
    # FP32 accumulation of 2^20 BF16 products per entry
    assert rel_fro(SA.cpu().numpy()[rows], ref, np.linalg.norm(ref)) <= 1e-6
    assert rel_fro(Sb.cpu().numpy()[rows], refb, np.linalg.norm(refb)) <= 1e-6


def test_full_size_srht_sampled_rows(problem):
    A, b = problem
    c = ctx()
    SA, Sb = c.sketch(dev(A), dev(b), D, kind="srht", seed=1)
    rows = [0, 1, 511, 1023]
    ref = OS.srht_rows(A, D, 1, rows)
    refb = OS.srht_rows(b, D, 1, rows)
    scale = np.linalg.norm(ref)
    assert rel_fro(SA.cpu().numpy()[rows], ref, scale) <= 1e-6
    assert rel_fro(Sb.cpu().numpy()[rows], refb, np.linalg.norm(refb)) <= 1e-6
