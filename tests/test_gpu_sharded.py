"""Row-sharded sketching on one GPU: the sketches of row blocks taken at their
global indices (snsolve_sketch_rows) sum to the sketch of the whole matrix, and
the replicated solve of a given [SA | Sb] (snsolve_solve_sketched) is the
solve snsolve_lstsq runs.  On integer-valued data with the bucket-sorted
CountSketch every partial sum is exact, so the match is bit for bit; the
float-reduction sketches (streaming CountSketch, sparse sign, Gaussian) match
within their parity tolerances."""
import numpy as np
import pytest
import torch

from gpu_util import ctx, dev

pytestmark = pytest.mark.gpu

M, N, D = 100003, 64, 256
CUTS = [0, 33336, 70000, M]          # multiples of 8 (the Gaussian's hash serves 8 rows)


def _int_problem():
    rng = np.random.default_rng(5)
    A = rng.integers(-8, 9, size=(M, N)).astype(np.float32)
    b = rng.integers(-8, 9, size=M).astype(np.float32)
    return A, b


def _parts_sum(c, Ad, bd, kind, variant):
    SA = torch.zeros((D, N), dtype=torch.float64, device="cuda")
    Sb = torch.zeros(D, dtype=torch.float64, device="cuda")
    for r0, r1 in zip(CUTS, CUTS[1:]):
        pa, pb = c.sketch_rows(Ad[r0:r1], bd[r0:r1], r0, D, kind=kind, seed=3, variant=variant)
        SA += pa.double()
        Sb += pb.double()
    return SA.cpu().numpy(), Sb.cpu().numpy()


def test_sorted_countsketch_parts_sum_exactly():
    c = ctx()
    A, b = _int_problem()
    Ad, bd = dev(A), dev(b)
    SA, Sb = c.sketch(Ad, bd, D, seed=3, variant="sorted")
    pSA, pSb = _parts_sum(c, Ad, bd, "countsketch", "sorted")
    assert np.array_equal(pSA, SA.cpu().numpy().astype(np.float64))
    assert np.array_equal(pSb, Sb.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("kind,variant,tol", [("countsketch", "stream", 1e-6), ("sparse_sign", "4", 1e-6),
                                              ("gaussian", "auto", 1e-6)])
def test_float_reduction_sketches_parts_sum(kind, variant, tol):
    c = ctx()
    rng = np.random.default_rng(6)
    A = rng.standard_normal((M, N)).astype(np.float32)
    b = rng.standard_normal(M).astype(np.float32)
    Ad, bd = dev(A), dev(b)
    SA, Sb = c.sketch(Ad, bd, D, kind=kind, seed=3, variant=variant)
    pSA, pSb = _parts_sum(c, Ad, bd, kind, variant)
    full = np.column_stack([SA.cpu().numpy(), Sb.cpu().numpy()]).astype(np.float64)
    part = np.column_stack([pSA, pSb])
    assert np.linalg.norm(part - full) / np.linalg.norm(full) <= tol


def test_srht_rows_rejected():
    import ctypes as C
    import paper_2409_14309_gb300 as sns
    from paper_2409_14309_gb300 import abi
    c = ctx()
    A, b = _int_problem()
    Ad, bd = dev(A[:1000]), dev(b[:1000])
    prob, sk = sns.dense_problem(Ad, bd), sns.sketch_desc(64, "srht", 1)
    SA = torch.empty((64, N), device="cuda")
    Sb = torch.empty(64, device="cuda")
    code = abi.lib().snsolve_sketch_rows(c.h, C.byref(prob), C.byref(sk), 0, C.c_void_p(SA.data_ptr()), N,
                                         C.c_void_p(Sb.data_ptr()), None, 0, None)
    assert code == abi.SNS_EINVAL


@pytest.mark.parametrize("n", [16, 64])
def test_solve_sketched_is_the_lstsq_solve(n):
    """snsolve_lstsq's sketch-and-solve (sorted CountSketch: reproducible) and
    snsolve_solve_sketched on the same [SA | Sb] give the same x^ bit for bit."""
    c = ctx()
    rng = np.random.default_rng(n)
    A = rng.standard_normal((20000, n)).astype(np.float32)
    b = rng.standard_normal(20000).astype(np.float32)
    Ad, bd = dev(A), dev(b)
    x1, i1 = c.lstsq(Ad, bd, 4 * n, seed=8, variant="sorted")
    SA, Sb = c.sketch(Ad, bd, 4 * n, seed=8, variant="sorted")
    x2, i2 = c.solve_sketched(torch.cat([SA, Sb[:, None]], 1).contiguous())
    assert i1.status == 0 and i2.status == 0
    assert torch.equal(x1, x2)
    assert i1.sketch_resid == i2.sketch_resid
