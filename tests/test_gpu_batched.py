"""Batched sketch-and-solve (one persistent launch over uneven problems) on the
GPU vs the FP64 oracle, problem by problem."""
import os

import numpy as np
import pytest
import torch

from gpu_util import ctx, dev
from oracle import sketch as OS
from oracle import solve as OL
from synth import ill_conditioned_problem

pytestmark = pytest.mark.gpu


def _xhat_tol(SA_ref):
    s = np.linalg.svd(SA_ref, compute_uv=False)
    return max(1e-5, 10 * (s[0] / s[-1]) * 2.0 ** -24)


def _batch(nprob, seed, m_lo, m_hi, ns, dfac=4, pad_every=5):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(nprob):
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.choice(ns))
        A, b, _ = ill_conditioned_problem(m, n, seed=seed * 1000 + i, kappa=1e3, noise=1e-3)
        d = dfac * n + (i % 3)                      # mostly 4n, some not
        pad = 3 if i % pad_every == 0 else 0
        probs.append((A, b, d, 17 + i, pad))
    return probs


def _to_dev(probs):
    As, bs = [], []
    for A, b, d, s, pad in probs:
        Af = np.zeros((A.shape[0], A.shape[1] + pad), dtype=np.float32)
        Af[:, :A.shape[1]] = A
        As.append(dev(Af)[:, :A.shape[1]])
        bs.append(dev(b))
    return As, bs


def test_batched_matches_oracle_per_problem(tmp_path, monkeypatch):
    monkeypatch.setenv("SNSOLVE_TUNE_CACHE", str(tmp_path / "tune.txt"))
    c = ctx()
    c._L.snsolve_tune_reset()
    probs = _batch(48, 1, 200, 6000, [1, 4, 16, 33, 64, 128])
    As, bs = _to_dev(probs)
    xs, infos = c.lstsq_batched(As, bs, [p[2] for p in probs], [p[3] for p in probs])
    torch.cuda.synchronize()
    for (A, b, d, seed, _), x, info in zip(probs, xs, infos):
        assert info.status == 0
        SA, Sb = OS.countsketch_apply(A, d, seed), OS.countsketch_apply(b, d, seed)
        x_ref, _, rn = OL.sketch_and_solve(SA, Sb)
        err = np.linalg.norm(x.cpu().numpy() - x_ref) / np.linalg.norm(x_ref)
        assert err <= _xhat_tol(SA), (A.shape, d, err)
        assert abs(info.sketch_resid - rn) <= 1e-5 * max(rn, 1e-30) + 1e-6 * np.linalg.norm(Sb)
    # the tuner measured this batch shape and wrote it to the cache file
    assert (tmp_path / "tune.txt").exists() and "batched:" in (tmp_path / "tune.txt").read_text()
    # replay (graph path, tuned shape from cache) gives the same answers within FP32 rounding
    xs2, infos2 = c.lstsq_batched(As, bs, [p[2] for p in probs], [p[3] for p in probs])
    for x1, x2, (A, b, d, seed, _) in zip(xs, xs2, probs):
        SA = OS.countsketch_apply(A, d, seed)
        assert torch.linalg.norm(x1 - x2) / torch.linalg.norm(x1) <= _xhat_tol(SA)


def test_batched_rank_deficient_member_flagged():
    c = ctx()
    rng = np.random.default_rng(3)
    As, bs, ds = [], [], []
    for i in range(6):
        A = rng.standard_normal((3000, 8)).astype(np.float32)
        if i == 2:
            A[:, 7] = A[:, 0]
        As.append(dev(A))
        bs.append(dev(rng.standard_normal(3000).astype(np.float32)))
        ds.append(32)
    xs, infos = c.lstsq_batched(As, bs, ds, list(range(6)))
    assert [i.status for i in infos] == [0, 0, 3, 0, 0, 0]


def test_batched_config4_shapes_sampled():
    """Shapes of the batched workload (m in [4096, 65536], n in {16,32,64,128},
    d = 4n, kappa 1e3) on a 96-problem batch; 12 problems checked against the oracle."""
    c = ctx()
    rng = np.random.default_rng(44)
    probs = []
    for i in range(96):
        m = int(rng.integers(4096, 65537))
        n = int(rng.choice([16, 32, 64, 128]))
        A, b, _ = ill_conditioned_problem(m, n, seed=5000 + i, kappa=1e3, noise=1e-3)
        probs.append((A, b, 4 * n, 1, 0))
    As, bs = _to_dev(probs)
    xs, infos = c.lstsq_batched(As, bs, [p[2] for p in probs], [p[3] for p in probs])
    assert all(i.status == 0 for i in infos)
    for j in range(0, 96, 8):
        A, b, d, seed, _ = probs[j]
        SA, Sb = OS.countsketch_apply(A, d, seed), OS.countsketch_apply(b, d, seed)
        x_ref, _, _ = OL.sketch_and_solve(SA, Sb)
        err = np.linalg.norm(xs[j].cpu().numpy() - x_ref) / np.linalg.norm(x_ref)
        assert err <= _xhat_tol(SA), (j, err)


def test_batched_rejects_unsupported_options():
    import ctypes as C
    import paper_2409_14309_gb300 as sns
    c = ctx()
    A = dev(np.ones((100, 4), dtype=np.float32))
    b = dev(np.ones(100, dtype=np.float32))
    probs = (sns.abi.sns_problem * 1)(sns.dense_problem(A, b))
    ops = (sns.abi.sns_opts * 1)(sns.opts(16, "countsketch", 1, tol=1e-8))
    n = C.c_size_t()
    assert c._L.snsolve_lstsq_batched_workspace_size(probs, ops, 1, C.byref(n)) == 0
    xp = (C.c_void_p * 1)(torch.empty(4, dtype=torch.float64, device="cuda").data_ptr())
    ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    code = c._L.snsolve_lstsq_batched(c.h, probs, ops, 1, xp, None, C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert code == 1      # tol > 0 is for snsolve_lstsq, not the batched sketch-and-solve
