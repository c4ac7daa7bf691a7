"""Sketch-and-apply (SAA-SAS, Sec. 2.1) on the GPU against the FP64 oracle.

The explicit Y = A R^-1 is checked entry by entry against the oracle's
apply_inverse_r (the same R, taken from the oracle's QR of the oracle's
sketch), within the deterministic error bound of an FP32 (or FP64) product:
|fl(A R^-1) - A R^-1| <= gamma_{n+1} |A| |R^-1| componentwise (the +1 covers
rounding R^-1 to FP32).  The solves are checked by what pins them: eta <= tol
computed by the oracle in FP64, and, run to the floor, the oracle's
sketch_and_apply answer x* (its fixed point, pinned to the Householder x*)."""
import numpy as np
import pytest
import torch

from gpu_util import ctx, dev
from oracle import sketch as OS
from oracle import solve as OL
from synth import ill_conditioned_problem

pytestmark = pytest.mark.gpu

U32, U64 = 2.0 ** -24, 2.0 ** -53


@pytest.mark.parametrize("m,n,dtype", [(5000, 37, np.float32), (70001, 256, np.float32), (3001, 300, np.float32),
                                       (4099, 64, np.float64)])
def test_form_y_matches_oracle(m, n, dtype):
    from paper_2409_14309_gb300 import abi
    import paper_2409_14309_gb300 as sns
    import ctypes as C
    ctx()
    A, b, _ = ill_conditioned_problem(m, n, seed=m + n, kappa=1e4, noise=1e-3, dtype=dtype)
    A64 = A.astype(np.float64)
    d = 4 * n
    _, R, _ = OL.sketch_and_solve(OS.countsketch_apply(A64, d, 2), OS.countsketch_apply(b.astype(np.float64), d, 2))
    Rinv = np.linalg.inv(R)                                   # upper triangular up to rounding
    Rinv = np.triu(Rinv)
    Ad, bd = dev(A), dev(b)
    prob = sns.dense_problem(Ad, bd)
    ldy = n + 3
    Y = torch.full((m, ldy), float("nan"), dtype=Ad.dtype, device="cuda")
    Rd = dev(Rinv)
    code = abi.lib().snsolve_debug_form_y(C.byref(prob), C.c_void_p(Rd.data_ptr()), C.c_void_p(Y.data_ptr()), ldy,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    Yg = Y.cpu().numpy()[:, :n].astype(np.float64)
    Y_ref = OL.apply_inverse_r(A64, R)
    u = U32 if dtype == np.float32 else U64
    gamma = (n + 1) * u / (1 - (n + 1) * u)
    # the R^-1 handed to the kernel is itself inexact: A Rinv - A R^-1 = A E R^-1 with
    # E = Rinv R - I (bounded by its FP64 value plus its own rounding)
    Ea = np.abs(Rinv @ R - np.eye(n)) + n * U64 * (np.abs(Rinv) @ np.abs(R))
    bound = (gamma * (np.abs(A64) @ np.abs(Rinv)) + np.abs(A64) @ (Ea @ np.abs(Rinv))
             + 1e3 * U64 * np.abs(Y_ref))                    # + the oracle's own FP64 rounding
    excess = np.abs(Yg - Y_ref) - bound
    assert np.all(np.isfinite(Yg))
    assert excess.max() <= 0.0, excess.max()
    print(f"m={m} n={n} {np.dtype(dtype).name}: |Y - Y_ref|_F / |Y_ref|_F = "
          f"{np.linalg.norm(Yg - Y_ref) / np.linalg.norm(Y_ref):.2e}")


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_saa_reaches_tol(tol):
    c = ctx()
    A, b, _ = ill_conditioned_problem(65536, 64, seed=11, kappa=1e6, noise=1e-4)
    x, info = c.lstsq(dev(A), dev(b), 256, seed=1, tol=tol, method="saa")
    assert info.status == 0, info.status
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    eta = OL.eta(A64, b64, x.cpu().numpy())
    print(f"SAA tol {tol:g}: eta {eta:.3e} (reported {info.eta:.3e}), {info.iters} passes over Y, "
          f"{info.outer} residual passes")
    assert eta <= tol * 1.5, (eta, info.eta)
    assert abs(info.eta - eta) <= 0.05 * eta + 2e-11


@pytest.mark.parametrize("dtype,kappa", [(np.float32, 1e6), (np.float64, 1e8)])
def test_saa_forward_error_at_floor_matches_oracle_saa(dtype, kappa):
    """Run to the floor, the GPU's SAA answer equals the oracle's SAA-SAS
    answer (both x*) to the perturbation bound kappa * u64."""
    c = ctx()
    A, b, _ = ill_conditioned_problem(40000, 48, seed=21, kappa=kappa, noise=1e-4, dtype=dtype)
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    x, info = c.lstsq(dev(A), dev(b), 192, seed=3, tol=1e-13, max_iter=600, method="saa")
    SA, Sb = OS.countsketch_apply(A64, 192, 3), OS.countsketch_apply(b64, 192, 3)
    x_saa, _, _, _ = OL.sketch_and_apply(A64, b64, SA, Sb, tol=1e-15, max_iter=400)
    err = np.linalg.norm(x.cpu().numpy() - x_saa) / np.linalg.norm(x_saa)
    print(f"SAA {np.dtype(dtype).name} kappa {kappa:g}: forward error vs oracle SAA {err:.3e} "
          f"(status {info.status}, {info.iters} passes)")
    assert err <= 100 * kappa * U64, err


def test_saa_and_sap_agree():
    """Both methods converge to the same least-squares solution."""
    c = ctx()
    A, b, _ = ill_conditioned_problem(100000, 128, seed=31, kappa=1e5, noise=1e-4)
    xa, ia = c.lstsq(dev(A), dev(b), 512, seed=4, tol=1e-10, method="saa")
    xp, ip = c.lstsq(dev(A), dev(b), 512, seed=4, tol=1e-10, method="sap")
    assert ia.status == 0 and ip.status == 0
    xa, xp = xa.cpu().numpy(), xp.cpu().numpy()
    assert np.linalg.norm(xa - xp) / np.linalg.norm(xp) <= 1e-10 * 1e5 * 10
