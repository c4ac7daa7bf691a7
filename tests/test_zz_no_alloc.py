"""The allocation-free CountSketch entry point, checked against snsolve_sketch.

Callers that cannot allocate device memory (inside host callbacks, under
allocators frozen after start-up, or with all device memory reserved up front)
use snsolve_sketch_countsketch_static, whose scratch is a fixed array inside
the library.  Two calls in a row must each give the same SA and Sb as the
workspace-based entry point, within the CountSketch tolerance used elsewhere.
This file is collected last so that a failure here does not hide other tests."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_util import ctx, dev, rel_fro

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


def _static_call(prob, d, seed, SA, Sb):
    from paper_2409_14309_gb300 import abi
    return abi.lib().snsolve_sketch_countsketch_static(
        C.byref(prob), d, seed, C.c_void_p(SA.data_ptr()), SA.stride(0), C.c_void_p(Sb.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("m,n,d", [(200003, 64, 256), (65536, 257, 1024)])
def test_static_scratch_matches_workspace_entry_point(m, n, d):
    import paper_2409_14309_gb300 as sns
    c = ctx()
    rng = np.random.default_rng(m + n)
    A = dev(rng.standard_normal((m, n)).astype(np.float32))
    b = dev(rng.standard_normal(m).astype(np.float32))
    ref_SA, ref_Sb = c.sketch(A, b, d, seed=11, variant="sorted")
    prob = sns.dense_problem(A, b)
    scale = float(torch.sqrt(torch.sum(A.double() ** 2) + torch.sum(b.double() ** 2)))
    for _ in range(2):                     # two calls in a row share the scratch
        SA = torch.full((d, n), float("nan"), device="cuda")
        Sb = torch.full((d,), float("nan"), device="cuda")
        assert _static_call(prob, d, 11, SA, Sb) == 0
        torch.cuda.synchronize()
        assert rel_fro(SA.cpu().numpy(), ref_SA.cpu().numpy(), scale) <= TOL32
        assert rel_fro(Sb.cpu().numpy(), ref_Sb.cpu().numpy(), scale) <= TOL32


def test_static_scratch_rejects_oversize_problem():
    """A 2^23-row problem needs about 32 MiB of scratch: rejected with
    SNS_ENOMEM before any launch.  The buffers are real (128 MiB of A), so the
    call would stay in bounds even if the size check were missing."""
    import paper_2409_14309_gb300 as sns
    ctx()
    m, n, d = 1 << 23, 4, 16
    A = torch.zeros((m, n), device="cuda")
    b = torch.zeros(m, device="cuda")
    prob = sns.dense_problem(A, b)
    SA = torch.full((d, n), 7.0, device="cuda")
    Sb = torch.full((d,), 7.0, device="cuda")
    assert _static_call(prob, d, 1, SA, Sb) == 2       # SNS_ENOMEM
    torch.cuda.synchronize()
    assert bool(torch.all(SA == 7.0)) and bool(torch.all(Sb == 7.0))   # nothing was written
