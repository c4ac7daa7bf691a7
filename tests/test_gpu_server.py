"""The request server: results equal to solving alone, HBM-budget admission,
bounded polls."""
import threading
import time

import numpy as np
import pytest
import torch

from gpu_util import ctx, dev
from oracle import solve as OL
from synth import csr_problem, ill_conditioned_problem

pytestmark = pytest.mark.gpu


def _mixed_requests():
    reqs = []
    shapes = [(20000, 32, 0.0), (70000, 64, 1e-3), (150000, 128, 1e-10), (5000, 8, 0.0), (300000, 256, 1e-10),
              (40000, 96, 1e-3), (90000, 33, 0.0)]
    for i, (m, n, tol) in enumerate(shapes):
        A, b, _ = ill_conditioned_problem(m, n, seed=700 + i, kappa=1e4, noise=1e-3)
        reqs.append(("dense", dev(A), dev(b), n, 4 * n, 11 + i, tol, A, b))
    for i, (m, n, dens, tol) in enumerate([(60000, 64, 0.05, 1e-3), (120000, 128, 0.02, 1e-10)]):
        A, b, _ = csr_problem(m, n, seed=800 + i, density=dens, n_dense=8)
        reqs.append(("csr", (dev(A.rowptr), dev(A.col), dev(A.val)), dev(b), n, 4 * n, 21 + i, tol, A, b))
    return reqs


def test_results_same_alone_and_in_the_mix():
    import paper_2409_14309_gb300 as sns
    c = ctx()
    reqs = _mixed_requests()
    # alone, one at a time
    alone = []
    for kind, A, b, n, d, seed, tol, _, _ in reqs:
        if kind == "dense":
            x, info = c.lstsq(A, b, d, seed=seed, tol=tol)
        else:
            x, info = c.lstsq_csr(*A, b, n, d, seed=seed, tol=tol, variant="sorted")
        assert info.status == 0
        alone.append(x.clone())
    # in the mix: all submitted at once to a 4-slot server
    srv = sns.Server(c, hbm_budget_bytes=16 << 30, max_slots=4)
    ids = []
    for kind, A, b, n, d, seed, tol, _, _ in reqs:
        if kind == "dense":
            ids.append(srv.submit(A, b, d, seed=seed, tol=tol))
        else:
            ids.append(srv.submit_csr(*A, b, n, d, seed=seed, tol=tol, variant="sorted"))
    for (rid, x), xa, (kind, _, _, n, d, seed, tol, Ah, bh) in zip(ids, alone, reqs):
        code, info = srv.poll(rid, timeout_us=120_000_000)
        assert code == 0 and info.status == 0
        # dense solves and CSR solves with variant "sorted" are reproducible:
        # the same bits alone and in the mix
        assert torch.equal(x, xa), kind
        if kind == "csr" and tol > 0:
            assert OL.eta(Ah.to_dense(), bh.astype(np.float64), x.cpu().numpy()) <= 1.5 * tol
    srv.close()


def test_request_over_budget_refused():
    import paper_2409_14309_gb300 as sns
    c = ctx()
    srv = sns.Server(c, hbm_budget_bytes=1 << 20, max_slots=2)
    A = torch.randn(20000, 64, device="cuda")
    b = torch.randn(20000, device="cuda")
    with pytest.raises(sns.SnsError) as e:
        srv.submit(A, b, 256)
    assert e.value.code == 8        # SNS_EBUDGET
    srv.close()


def test_admission_never_exceeds_budget():
    import paper_2409_14309_gb300 as sns
    c = ctx()
    m, n = 200000, 128
    A = torch.randn(m, n, device="cuda")
    b = torch.randn(m, device="cuda")
    prob = sns.dense_problem(A, b)
    op = sns.opts(512, "countsketch", 1, tol=1e-8)
    ws = c.lstsq_workspace(prob, op)
    foot = m * n * 4 + m * 4 + ((ws + 255) // 256) * 256
    budget = 3 * foot + foot // 2                 # room for three requests at a time
    srv = sns.Server(c, hbm_budget_bytes=budget, max_slots=8)
    peak = {"used": 0, "running": 0}
    stop = threading.Event()

    def watch():
        while not stop.is_set():
            r, p, u = srv.stats()
            peak["used"] = max(peak["used"], u)
            peak["running"] = max(peak["running"], r)
            time.sleep(0.0002)

    t = threading.Thread(target=watch)
    t.start()
    ids = [srv.submit(A, b, 512, seed=i, tol=1e-8)[0] for i in range(12)]
    for rid in ids:
        code, info = srv.poll(rid, timeout_us=120_000_000)
        assert code == 0 and info.status == 0
    stop.set()
    t.join()
    srv.close()
    assert peak["used"] <= budget
    assert 1 <= peak["running"] <= 3


def test_poll_timeout_and_eagain_and_unknown_id():
    import paper_2409_14309_gb300 as sns
    c = ctx()
    srv = sns.Server(c, hbm_budget_bytes=16 << 30, max_slots=1)
    big_A = torch.randn(1 << 20, 256, device="cuda")
    big_b = torch.randn(1 << 20, device="cuda")
    small_A = torch.randn(5000, 16, device="cuda")
    small_b = torch.randn(5000, device="cuda")
    rid_big, _ = srv.submit(big_A, big_b, 1024, tol=1e-12, max_iter=200)
    rid_small, _ = srv.submit(small_A, small_b, 64)
    code, _ = srv.poll(rid_small, timeout_us=0)
    assert code == 5            # SNS_EAGAIN: queued behind the big request on the single slot
    code, _ = srv.poll(rid_small, timeout_us=200)
    assert code == 6            # SNS_ETIMEOUT after a bounded wait
    for rid in (rid_big, rid_small):
        code, info = srv.poll(rid, timeout_us=120_000_000)
        assert code == 0
    code, _ = srv.poll(rid_small, timeout_us=0)
    assert code == 1            # collected already: unknown id
    srv.close()


def test_small_request_overtakes_one_waiting_for_memory():
    """Two slots, budget for one large request plus small ones: while the first
    large request runs, the second must wait for memory, and a small request
    submitted after it is admitted ahead of it and finishes first."""
    import paper_2409_14309_gb300 as sns
    c = ctx()
    m, n = 1 << 21, 256
    A1 = torch.randn(m, n, device="cuda")
    b1 = torch.randn(m, device="cuda")
    A2 = torch.randn(m, n, device="cuda")
    b2 = torch.randn(m, device="cuda")
    As = torch.randn(5000, 16, device="cuda")
    bs = torch.randn(5000, device="cuda")
    prob = sns.dense_problem(A1, b1)
    op = sns.opts(1024, "countsketch", 1, tol=1e-12, max_iter=200)
    foot = m * n * 4 + m * 4 + ((c.lstsq_workspace(prob, op) + 255) // 256) * 256
    srv = sns.Server(c, hbm_budget_bytes=foot + foot // 4, max_slots=2)
    rid1, _ = srv.submit(A1, b1, 1024, seed=1, tol=1e-12, max_iter=200)
    rid2, _ = srv.submit(A2, b2, 1024, seed=2, tol=1e-12, max_iter=200)
    rids, _ = srv.submit(As, bs, 64, seed=3)
    code, info = srv.poll(rids, timeout_us=60_000_000)
    assert code == 0 and info.status == 0
    # the small request ran beside the first large one: that one has not finished
    # yet (in strict arrival order the small one would have waited for the second
    # large one's admission, which follows the first one's completion)
    code1, _ = srv.poll(rid1, timeout_us=0)
    assert code1 == 5               # SNS_EAGAIN
    code2, _ = srv.poll(rid2, timeout_us=0)
    assert code2 == 5
    for rid in (rid1, rid2):
        code, info = srv.poll(rid, timeout_us=120_000_000)
        assert code == 0
    srv.close()
