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


def test_full_size_gaussian_sampled_rows(problem):
    A, b = problem
    c = ctx()
    SA, Sb = c.sketch(dev(A), dev(b), D, kind="gaussian", seed=1)
    rows = [0, 7, 8, 31, 32, 500, 1023]
    ref = OS.gaussian_rows(A, D, 1, rows)
    refb = OS.gaussian_rows(b, D, 1, rows)
    # FP32 accumulation of 2^20 BF16 products per entry
    assert rel_fro(SA.cpu().numpy()[rows], ref, np.linalg.norm(ref)) <= 1e-5
    assert rel_fro(Sb.cpu().numpy()[rows], refb, np.linalg.norm(refb)) <= 1e-5


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
