"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_ctx = None


def ctx():
    global _ctx
    need_gpu()
    if _ctx is None:
        import paper_2409_14309_gb300 as sns
        _ctx = sns.Context(0)
    return _ctx


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel_fro(a, b, scale):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) / scale)
