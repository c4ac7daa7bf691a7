"""The paper's benchmark generator (Sec. 3.1, after Epperly et al. 2024):
what its construction fixes, checked with independent library routines."""
import numpy as np

from oracle import solve as OL
from synth import paper_problem


def test_paper_problem_closed_form():
    m, n, kappa, beta = 3000, 40, 1e10, 1e-10
    A, b, x_star = paper_problem(m, n, seed=5, kappa=kappa, beta=beta)
    s = np.linalg.svd(A, compute_uv=False)                     # LAPACK
    assert np.isclose(s[0], 1.0, rtol=1e-12) and np.isclose(s[0] / s[-1], kappa, rtol=1e-4)
    assert np.isclose(np.linalg.norm(x_star), 1.0, rtol=1e-14)
    r = b - A @ x_star
    assert np.isclose(np.linalg.norm(r), beta, rtol=1e-5)
    # r* is orthogonal to range(A): A^T r* is at the rounding level of forming b
    assert np.linalg.norm(A.T @ r) <= 1e-15 * np.sqrt(m)
    # the oracle's Householder least-squares solution is x* to kappa * u64
    x, rn = OL.exact_lstsq(A, b)
    assert np.linalg.norm(x - x_star) <= 1e3 * kappa * 2.0 ** -53
