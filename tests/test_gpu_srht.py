"""SRHT apply on the GPU vs the FP64 oracle (Sec. 1.2.1: Hadamard-based sketch
with a fast transform, S = (1/sqrt(d)) P H D on [A | b] padded
to m' = 2^ceil(log2 m) rows).  SA and Sb within ||SA_gpu - SA_ref||_F /
||[A | b]||_F <= 1e-6 for FP32 data (1e-13 for FP64 data).  Each output row is
a signed sum over all m' rows, so a wrong sampled row or sign shows up as an
O(1) relative error, not a rounding one.  The cases cover both samplers
(shared-memory bitmap for m' <= 2^20, hash set above), the one-pass FP32 form
(m' >= 1024, d <= 1024, with and without a b-only column tile, aligned and
unaligned rows), the two-pass forms (d > 1024; m' < 1024; FP64), ragged m and
d = m'."""
import numpy as np
import pytest

from gpu_util import ctx, dev, rel_fro
from oracle import sketch as OS

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


@pytest.mark.parametrize("m,n,d", [
    (5, 2, 3), (1000, 7, 64), (1024, 8, 1024), (3000, 16, 128), (70000, 33, 500), (131072, 64, 2048),
    ((1 << 20) + 3, 4, 256),
])
def test_srht_dense_f32(m, n, d):
    c = ctx()
    rng = np.random.default_rng(m + 31 * n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal(m).astype(np.float32)
    SA, Sb = c.sketch(dev(A), dev(b), d, kind="srht", seed=m % 97)
    scale = np.sqrt(np.linalg.norm(A.astype(np.float64)) ** 2 + np.linalg.norm(b.astype(np.float64)) ** 2)
    assert rel_fro(SA.cpu().numpy(), OS.srht_apply(A, d, m % 97), scale) <= TOL32
    assert rel_fro(Sb.cpu().numpy(), OS.srht_apply(b, d, m % 97), scale) <= TOL32


@pytest.mark.parametrize("m,n,d,pad", [(5000, 31, 200, 0), (70001, 47, 300, 3), (20000, 256, 1024, 1)])
def test_srht_one_pass_tiles_and_strides(m, n, d, pad):
    """The one-pass FP32 form (m' >= 1024, d <= 1024): n + 1 a multiple of the
    16-column tile (no b-only tile), and rows padded so that lda is not a
    multiple of 4 (element loads instead of float4) with a partial last tile."""
    import torch
    c = ctx()
    rng = np.random.default_rng(m + n + pad)
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal(m).astype(np.float32)
    big = torch.zeros((m, n + pad), dtype=torch.float32, device="cuda")
    big[:, :n] = dev(A)
    Ad = big[:, :n]
    assert Ad.stride(0) == n + pad
    SA, Sb = c.sketch(Ad, dev(b), d, kind="srht", seed=7)
    scale = np.sqrt(np.linalg.norm(A.astype(np.float64)) ** 2 + np.linalg.norm(b.astype(np.float64)) ** 2)
    assert rel_fro(SA.cpu().numpy(), OS.srht_apply(A, d, 7), scale) <= TOL32
    assert rel_fro(Sb.cpu().numpy(), OS.srht_apply(b, d, 7), scale) <= TOL32
    # bitwise repeatable: fixed block order inside a CTA, CTA order in the reduction
    SA2, Sb2 = c.sketch(Ad, dev(b), d, kind="srht", seed=7)
    assert torch.equal(SA, SA2) and torch.equal(Sb, Sb2)


@pytest.mark.parametrize("m,n,d", [(9, 3, 4), (4097, 10, 100)])
def test_srht_dense_f64(m, n, d):
    c = ctx()
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    SA, Sb = c.sketch(dev(A), dev(b), d, kind="srht", seed=5)
    scale = np.linalg.norm(np.column_stack([A, b]))
    assert rel_fro(SA.cpu().numpy(), OS.srht_apply(A, d, 5), scale) <= 1e-13
    assert rel_fro(Sb.cpu().numpy(), OS.srht_apply(b, d, 5), scale) <= 1e-13


def test_srht_seeds_differ_and_repeat():
    """Same seed: the same sketch; another seed: another sample and signs."""
    c = ctx()
    rng = np.random.default_rng(2)
    A = dev(rng.standard_normal((5000, 12)).astype(np.float32))
    b = dev(rng.standard_normal(5000).astype(np.float32))
    s1 = c.sketch(A, b, 256, kind="srht", seed=1)[0].cpu().numpy()
    s1b = c.sketch(A, b, 256, kind="srht", seed=1)[0].cpu().numpy()
    s2 = c.sketch(A, b, 256, kind="srht", seed=2)[0].cpu().numpy()
    assert np.array_equal(s1, s1b)
    assert np.linalg.norm(s1 - s2) > 0.5 * np.linalg.norm(s1)


@pytest.mark.parametrize("mp,d", [
    (1, 1), (2, 2), (8, 8), (64, 60), (1024, 1000), (4096, 3000), (1 << 20, 1024), (1 << 20, 16384),
    (1 << 21, 1024), (1 << 30, 777),
])
def test_srht_row_sample_bit_exact(mp, d):
    """The sampled rows equal the oracle's Floyd sample exactly: dense cases
    (d close to m') make most draws collide and take the in-order path of the
    bitmap sampler; m' > 2^20 takes the hash-set sampler."""
    c = ctx()
    for seed in (0, 12345):
        got = c.srht_sample(mp, d, seed).cpu().numpy()
        assert np.array_equal(got, OS.srht_sample(mp, d, seed))


def test_srht_row_sample_rejects_out_of_range():
    """m' must be a power of two below 2^31 and 1 <= d <= m'."""
    import paper_2409_14309_gb300 as sns
    c = ctx()
    for mp, d in [(1 << 31, 8), (6, 2), (8, 9)]:
        with pytest.raises(sns.SnsError):
            c.srht_sample(mp, d, 0)
