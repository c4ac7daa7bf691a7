"""Pins of the oracle's sketch operators against definitions, closed forms and
independent library routines."""
import math

import numpy as np
import pytest
import torch
from scipy.special import ndtr

from oracle import hashing as H
from oracle import sketch as S
from oracle import solve as L


def test_countsketch_dense_equals_scatter_exactly():
    rng = np.random.default_rng(0)
    A = rng.integers(-50, 50, size=(333, 9)).astype(np.float64)
    for d in (1, 7, 64):
        Sm = S.countsketch_matrix(333, d, seed=11)
        assert np.array_equal(Sm @ A, S.countsketch_apply(A, d, 11))


def test_countsketch_structure_one_signed_entry_per_column():
    Sm = S.countsketch_matrix(500, 40, seed=2)
    assert np.array_equal(np.abs(Sm).sum(axis=0), np.ones(500))
    assert set(np.unique(Sm)) <= {-1.0, 0.0, 1.0}
    h, s = H.countsketch_hash(2, 500, 40)
    assert np.array_equal(Sm[h, np.arange(500)], s)


def test_countsketch_isometry_in_expectation():
    # E ||S x||^2 = ||x||^2 (E[S^T S] = I)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(400)
    vals = [np.linalg.norm(S.countsketch_apply(x, 32, seed)) ** 2 for seed in range(400)]
    se = np.std(vals) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - x @ x) < 4 * se


def test_countsketch_csr_equals_dense():
    from synth import csr_problem
    A, b, _ = csr_problem(300, 20, seed=4, density=0.2, n_dense=3)
    ref = S.countsketch_apply(A.to_dense(), 50, 9)
    got = S.countsketch_apply_csr(A.rowptr, A.col, A.val, A.n, 50, 9)
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.round_to_bf16_via_f32(x), ref)
    assert np.array_equal(S.round_to_bf16(x.astype(np.float64)), ref)


def test_gaussian_table_is_normal_quantiles():
    T = S.gaussian_table()
    n = T.size
    assert n == 256
    assert np.array_equal(T, -T[::-1])                           # symmetric
    assert np.all(np.diff(T) > 0)                                # strictly monotone
    # each entry is a BF16 number within half a BF16 ulp of the exact quantile:
    # Phi(T[j]) brackets (j + 1/2)/256 between the neighbouring BF16 values
    p = (np.arange(n) + 0.5) / n
    ulp = np.ldexp(1.0, np.frexp(T)[1] - 8)
    assert np.all(ndtr(T - ulp / 2) <= p + 1e-15)
    assert np.all(ndtr(T + ulp / 2) >= p - 1e-15)
    # 256 quantile midpoints: mean 0, second moment 1 - O(log(n) / n)
    assert abs(T.mean()) < 1e-12 and abs((T ** 2).mean() - 1) < 1e-2


def test_gaussian_indices_uniform_and_byte_layout():
    d, m = 10, 2003
    j = S.gaussian_indices(m, d, seed=5)
    assert j.shape == (d, m) and j.min() >= 0 and j.max() < 256
    counts = np.bincount(j.ravel() >> 2, minlength=64)           # 64 coarse bins
    e = j.size / 64
    assert ((counts - e) ** 2 / e).sum() < 64 + 6 * math.sqrt(128)
    # entry (k, i) is byte i mod 8 of output (i div 8) * d + k of stream 3
    for k, i in [(9, 7), (0, 0), (3, 2002), (5, 1608)]:
        key = int(H.splitmix64_at(H.stream_state(5, 3), np.array([(i // 8) * d + k], dtype=np.uint64))[0])
        assert j[k, i] == (key >> (8 * (i % 8))) & 0xFF
    # one output feeds the eight columns 8t .. 8t+7 of one row
    key = int(H.splitmix64_at(H.stream_state(5, 3), np.array([11 * d + 4], dtype=np.uint64))[0])
    assert [j[4, 88 + b] for b in range(8)] == [(key >> (8 * b)) & 0xFF for b in range(8)]


def test_gaussian_sketch_and_solve_expected_residual():
    # For Gaussian S with d > n + 1: E ||A x^ - b||^2 = (1 + n/(d-n-1)) ||A x* - b||^2.
    rng = np.random.default_rng(3)
    m, n, d = 1500, 8, 30
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    _, rn = L.exact_lstsq(A, b)
    ratios = []
    for seed in range(250):
        Sm = S.gaussian_matrix(m, d, seed)
        x, _, _ = L.sketch_and_solve(Sm @ A, Sm @ b)
        ratios.append(np.linalg.norm(A @ x - b) ** 2 / rn ** 2)
    expect = 1 + n / (d - n - 1)
    se = np.std(ratios) / math.sqrt(len(ratios))
    assert abs(np.mean(ratios) - expect) < 3.5 * se


def test_bf16_split_terms():
    """Three BF16 terms (8 significant bits each) hold an FP32 value exactly;
    two leave at most 2^-16 of it; each term is itself a BF16 number (torch's
    rounding leaves it unchanged), and every term after the first is at most
    2^-8 of the previous remainder's size."""
    rng = np.random.default_rng(12)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-40, 40, 200000))).astype(np.float32)
    x64 = x.astype(np.float64)
    parts = S.bf16_split(x, 3)
    for t in parts:
        assert np.array_equal(torch.from_numpy(t).to(torch.bfloat16).to(torch.float64).numpy(), t)
    assert np.array_equal(parts[0] + parts[1] + parts[2], x64)
    assert np.array_equal(S.bf16_terms(x, 3), x64)
    assert np.array_equal(S.bf16_terms(x, 1), torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy())
    assert np.all(np.abs(x64 - S.bf16_terms(x, 2)) <= np.ldexp(np.abs(x64), -16))
    assert np.all(np.abs(parts[1]) <= np.ldexp(np.abs(x64), -8))
    assert np.all(np.abs(parts[2]) <= np.ldexp(np.abs(x64 - parts[0]), -8))
    # one term is strictly coarser than two: most values are not BF16 numbers
    assert np.mean(S.bf16_terms(x, 1) != S.bf16_terms(x, 2)) > 0.9


def test_gaussian_apply_three_terms_is_exact_fp32():
    rng = np.random.default_rng(13)
    A = (rng.standard_normal((300, 6)) * np.exp(rng.uniform(-5, 5, (300, 6)))).astype(np.float32)
    Gm = S.gaussian_matrix(300, 16, 2)
    exact = Gm @ A.astype(np.float64)
    assert np.allclose(S.gaussian_apply(A, 16, 2, terms=3), exact, rtol=1e-13, atol=1e-13)
    assert np.allclose(S.gaussian_apply(A, 16, 2, bf16_operand=False), exact, rtol=1e-13, atol=1e-13)
    two = S.gaussian_apply(A, 16, 2, terms=2)
    assert np.abs(two - exact).max() <= 2.0 ** -16 * (np.abs(Gm) @ np.abs(A.astype(np.float64))).max()
    assert not np.allclose(S.gaussian_apply(A, 16, 2, terms=1), exact, rtol=1e-5, atol=0)


def test_gaussian_apply_bf16_operand():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((100, 5)).astype(np.float32)
    Ab = torch.from_numpy(A).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.allclose(S.gaussian_apply(A, 12, 1, bf16_operand=True), S.gaussian_matrix(100, 12, 1) @ Ab,
                       rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mp", [1, 2, 4, 64, 1024, 4096])
def test_hadamard_orthogonality(mp):
    Hm = S.hadamard_matrix(mp)
    assert np.array_equal(Hm @ Hm.T, mp * np.eye(mp))
    if mp >= 2:   # Sylvester recursion H_{2k} = [[H_k, H_k], [H_k, -H_k]]
        h = S.hadamard_matrix(mp // 2)
        assert np.array_equal(Hm, np.block([[h, h], [h, -h]]))


@pytest.mark.parametrize("mp", [1, 2, 8, 512, 2048])
def test_fwht_equals_explicit_product(mp):
    rng = np.random.default_rng(mp)
    X = rng.standard_normal((mp, 3))
    assert np.allclose(S.fwht(X), S.hadamard_matrix(mp) @ X, rtol=0, atol=1e-10)


def test_srht_sample_properties_and_uniformity():
    for (mp, d) in [(1, 1), (16, 16), (1024, 10), (1 << 20, 1024)]:
        P = S.srht_sample(mp, d, seed=3)
        assert P.size == d and np.all(np.diff(P) > 0) and P[0] >= 0 and P[-1] < mp
    # Floyd's algorithm: every d-subset equally likely (mp = 5, d = 2: 10 subsets)
    counts = {}
    for seed in range(5000):
        key = tuple(S.srht_sample(5, 2, seed))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 10
    c = np.array(list(counts.values()))
    assert ((c - 500) ** 2 / 500).sum() < 35          # chi2(9) far tail


@pytest.mark.parametrize("m", [1, 5, 64, 300])
def test_srht_fast_equals_dense(m):
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, 4))
    d = min(S.next_pow2(m), 16)
    assert np.allclose(S.srht_apply(A, d, 8), S.srht_matrix(m, d, 8) @ A, rtol=0, atol=1e-10)


def test_srht_isometry_in_expectation():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(200)
    vals = [np.linalg.norm(S.srht_apply(x, 32, seed)) ** 2 for seed in range(300)]
    se = np.std(vals) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - x @ x) < 4 * se


@pytest.mark.parametrize("m,n,d", [(1000, 5, 64), (4097, 3, 100)])
def test_single_row_forms_equal_the_full_sketches(m, n, d):
    """The one-row-at-a-time forms used to check full-size GPU results give the
    same rows as the full CountSketch, Gaussian and SRHT sketches (themselves
    pinned above: dense product = scatter, index layout, table quantiles, fast
    transform = dense product)."""
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n))
    rows = [0, 1, d // 2, d - 1]
    assert np.allclose(S.countsketch_rows(A, d, 4, rows), (S.countsketch_matrix(m, d, 4) @ A)[rows],
                       rtol=0, atol=1e-12)
    bb = rng.standard_normal(m)
    assert np.allclose(S.countsketch_rows(bb, d, 4, rows), (S.countsketch_matrix(m, d, 4) @ bb)[rows],
                       rtol=0, atol=1e-12)
    assert np.allclose(S.gaussian_rows(A, d, 5, rows), S.gaussian_apply(A, d, 5)[rows], rtol=0, atol=1e-12)
    assert np.allclose(S.gaussian_rows(A, d, 5, rows, bf16_operand=False),
                       S.gaussian_apply(A, d, 5, bf16_operand=False)[rows], rtol=0, atol=1e-12)
    assert np.allclose(S.srht_rows(A, d, 6, rows), S.srht_apply(A, d, 6)[rows], rtol=0, atol=1e-12)
    b = rng.standard_normal(m)
    assert np.allclose(S.srht_rows(b, d, 6, rows), S.srht_apply(b, d, 6)[rows], rtol=0, atol=1e-12)


# ---------------------------------------------------------------- sparse sign embedding

def test_sparse_sign_zeta1_is_the_countsketch():
    """With one nonzero per column the embedding is the CountSketch itself."""
    A = np.random.default_rng(1).standard_normal((3000, 4))
    assert np.array_equal(S.sparse_sign_apply(A, 77, 1, 9), S.countsketch_apply(A, 77, 9))


@pytest.mark.parametrize("zeta,d", [(2, 16), (4, 64), (8, 8), (3, 1000)])
def test_sparse_sign_structure(zeta, d):
    """Each column: exactly zeta nonzeros +-1/sqrt(zeta), at distinct rows; the
    scatter form equals the dense product."""
    m = 700
    Sm = S.sparse_sign_matrix(m, d, zeta, 4)
    nz = Sm != 0
    assert np.all(nz.sum(axis=0) == zeta)
    assert np.allclose(np.abs(Sm[nz]), 1 / math.sqrt(zeta))
    A = np.random.default_rng(zeta).standard_normal((m, 3))
    assert np.allclose(S.sparse_sign_apply(A, d, zeta, 4), Sm @ A, rtol=0, atol=1e-13)


def test_sparse_sign_rows_uniform_over_subsets():
    """Floyd's algorithm picks every zeta-subset of [0, d) with equal
    probability: d = 5, zeta = 2 gives 10 subsets, chi-square over 50000
    columns; the signs are balanced and independent of the rows."""
    from itertools import combinations
    rows, signs = S.sparse_sign_hash(50000, 5, 2, 11)
    keys = [tuple(sorted(r)) for r in rows]
    subsets = list(combinations(range(5), 2))
    counts = np.array([keys.count(c) for c in subsets], dtype=float)
    exp = 50000 / len(subsets)
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 27.9          # 9 degrees of freedom, p = 0.001
    assert abs(signs.mean()) < 0.02


def test_sparse_sign_isometry_in_expectation():
    """E ||S x||^2 = ||x||^2 (each column has zeta entries of square 1/zeta)."""
    x = np.random.default_rng(3).standard_normal(400)
    vals = [np.linalg.norm(S.sparse_sign_apply(x, 32, 4, seed)) ** 2 for seed in range(300)]
    assert abs(np.mean(vals) / np.linalg.norm(x) ** 2 - 1) < 0.05
