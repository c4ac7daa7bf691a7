"""The timeout path of a bounded device-side wait, forced without any fault.

The multi-CTA QR hands each Householder reflector between CTAs through device
memory, and every wait for one is bounded.  With the poll limit set to one, a
consumer gives up on the first reflector that is not yet published: the
kernel records its error word, finishes with zeros and returns, and
snsolve_lstsq reports SNS_ETIMEOUT.  The next solve at the default limit must
give the oracle's answer again (the context stays usable)."""
import numpy as np
import pytest

from gpu_util import ctx, dev

pytestmark = pytest.mark.gpu


def test_qr_wait_that_runs_out_reports_timeout_and_context_recovers():
    from oracle import sketch as OS
    from oracle import solve as OL
    from paper_2409_14309_gb300 import abi
    from synth import gaussian_problem
    import paper_2409_14309_gb300 as sns
    c = ctx()
    L = abi.lib()
    m, n, d = 8192, 96, 384                     # q = n + 1 >= 32: the multi-CTA QR
    A, b, _ = gaussian_problem(m, n, seed=41, noise=1e-3)
    Ad, bd = dev(A), dev(b)
    prob = sns.dense_problem(Ad, bd)
    op = sns.opts(d, "countsketch", 5)
    try:
        L.snsolve_debug_set_qr_wait_limit(1)
        for _ in range(2):
            _, info = c.lstsq_problem(prob, op, check=False)
            assert info.status == abi.SNS_ETIMEOUT, abi.status_name(info.status)
    finally:
        L.snsolve_debug_set_qr_wait_limit(0)
    x, info = c.lstsq_problem(prob, op)
    assert info.status == abi.SNS_OK
    x_ref, _, _ = OL.sketch_and_solve(OS.countsketch_apply(A, d, 5), OS.countsketch_apply(b, d, 5))
    assert np.linalg.norm(x.cpu().numpy() - x_ref) / np.linalg.norm(x_ref) < 1e-10
