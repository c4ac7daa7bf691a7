"""Host-side injected failures on the GPU path: each armed fault makes one call
fail with its documented status, the process and context stay usable, and the
next call gives the same result as a clean one.  No GPU faults, traps or hangs:
the failures are reported by host-side checks (the kernels that were launched
complete normally)."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_util import ctx, dev

pytestmark = pytest.mark.gpu


@pytest.fixture()
def L():
    from paper_2409_14309_gb300 import abi
    L = abi.lib()
    yield L
    L.snsolve_debug_set_fault(None)


def _problem(m=8192, n=64, seed=3):
    from synth import gaussian_problem
    A, b, _ = gaussian_problem(m, n, seed=seed, noise=1e-3)
    return A, b


def _raw_lstsq(c, prob, op):
    """snsolve_lstsq's return code and x (the binding's check bypassed)."""
    from paper_2409_14309_gb300 import abi
    import paper_2409_14309_gb300 as sns
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    need = c.lstsq_workspace(prob, op)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    info = abi.sns_info()
    code = c._L.snsolve_lstsq(c.h, C.byref(prob), C.byref(op), C.c_void_p(x.data_ptr()), C.byref(info),
                              C.c_void_p(ws.data_ptr()), ws.numel(), sns._stream(None))
    torch.cuda.synchronize()
    return code, x, info


def test_alloc_fault_fails_context_creation_once(L):
    from paper_2409_14309_gb300 import abi
    import paper_2409_14309_gb300 as sns
    ctx()                                                   # the shared context exists before arming
    assert L.snsolve_debug_set_fault(b"alloc") == abi.SNS_OK
    with pytest.raises(sns.SnsError) as e:
        sns.Context(0)
    assert e.value.code == abi.SNS_ENOMEM
    assert L.snsolve_last_cuda_error() == b"injected allocation failure"
    assert L.snsolve_debug_fault_armed(None) == 0           # fired once, disarmed
    c2 = sns.Context(0)                                     # the next creation succeeds
    assert c2.h


def test_alloc_fault_fails_server_creation_once(L):
    from paper_2409_14309_gb300 import abi
    import paper_2409_14309_gb300 as sns
    c = ctx()
    assert L.snsolve_debug_set_fault(b"alloc") == abi.SNS_OK
    with pytest.raises(sns.SnsError) as e:
        sns.Server(c, 1 << 30, 2)
    assert e.value.code == abi.SNS_ENOMEM
    s = sns.Server(c, 1 << 30, 2)
    del s


@pytest.mark.parametrize("nth", [1, 3, 6])
def test_launch_fault_stops_the_solve_and_the_next_solve_is_clean(L, nth):
    from paper_2409_14309_gb300 import abi
    import paper_2409_14309_gb300 as sns
    c = ctx()
    A, b = _problem()
    Ad, bd = dev(A).float(), dev(b).float()                # kept alive: the problem holds raw pointers
    prob = sns.dense_problem(Ad, bd)
    op = sns.opts(256, "countsketch", 11, tol=1e-8)
    code0, x0, info0 = _raw_lstsq(c, prob, op)
    assert code0 == abi.SNS_OK and info0.status == abi.SNS_OK
    assert L.snsolve_debug_set_fault(b"launch:%d" % nth) == abi.SNS_OK
    code, _, _ = _raw_lstsq(c, prob, op)
    assert code == abi.SNS_ECUDA, abi.status_name(code)
    assert L.snsolve_last_cuda_error() == b"injected launch failure"
    assert L.snsolve_debug_fault_armed(None) == 0
    code1, x1, info1 = _raw_lstsq(c, prob, op)
    assert code1 == abi.SNS_OK and info1.status == abi.SNS_OK
    assert torch.equal(x0, x1)                                # dense CountSketch SAP is bitwise repeatable


def test_timeout_fault_reports_expired_wait_and_the_next_solve_is_clean(L):
    from paper_2409_14309_gb300 import abi
    import paper_2409_14309_gb300 as sns
    c = ctx()
    A, b = _problem(seed=5)
    Ad, bd = dev(A).float(), dev(b).float()                # kept alive: the problem holds raw pointers
    prob = sns.dense_problem(Ad, bd)
    op = sns.opts(256, "countsketch", 13)
    code0, x0, _ = _raw_lstsq(c, prob, op)
    assert code0 == abi.SNS_OK
    assert L.snsolve_debug_set_fault(b"timeout") == abi.SNS_OK
    code, _, info = _raw_lstsq(c, prob, op)
    assert code == abi.SNS_ETIMEOUT and info.status == abi.SNS_ETIMEOUT
    code1, x1, _ = _raw_lstsq(c, prob, op)
    assert code1 == abi.SNS_OK
    assert torch.equal(x0, x1)


def test_timeout_fault_in_sketch_status(L):
    from paper_2409_14309_gb300 import abi
    import paper_2409_14309_gb300 as sns
    c = ctx()
    A, b = _problem(m=4096, n=32, seed=7)
    Ad, bd = dev(A).float(), dev(b).float()
    prob, sk = sns.dense_problem(Ad, bd), sns.sketch_desc(256, "gaussian", 3)
    need = c.sketch_workspace(prob, sk)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    c.sketch_problem(prob, sk, Ad.dtype, ws)
    st = sns._stream(None)
    assert L.snsolve_sketch_status(C.byref(prob), C.byref(sk), C.c_void_p(ws.data_ptr()), ws.numel(), st) == abi.SNS_OK
    assert L.snsolve_debug_set_fault(b"timeout") == abi.SNS_OK
    assert (L.snsolve_sketch_status(C.byref(prob), C.byref(sk), C.c_void_p(ws.data_ptr()), ws.numel(), st)
            == abi.SNS_ETIMEOUT)
    assert L.snsolve_sketch_status(C.byref(prob), C.byref(sk), C.c_void_p(ws.data_ptr()), ws.numel(), st) == abi.SNS_OK
