"""Sketch operators S in R^{d x m} and their application to [A | b] (steps 1-2 of the
sketch-and-solve paradigm, Sec. 1.2).  FP64 throughout.  TEST INFRASTRUCTURE ONLY.

Three families, as the paper lists them:

* Clarkson-Woodruff / CountSketch (Sec. 1.2.2, the paper's default): one nonzero
  per column of S, S[h(i), i] = s(i).  Reading: no scaling (E[S^T S] = I already,
  and a common scale does not change the minimiser).
* Gaussian (Sec. 1.2.1): S = G / sqrt(d) with G iid Gaussian.  Reading (the paper
  fixes no generator): G[k, i] = T[j], j an 8-bit index drawn from the hash
  stream, T[j] the BF16-rounded normal quantile Phi^{-1}((j + 1/2) / 256).  One
  SplitMix64 output of stream 3 serves eight consecutive columns of one row:
  entry (k, i) uses byte (i mod 8) of output (i div 8) * d + k.  The
  tensor-core path multiplies BF16 operands, so the oracle offers SA for both
  the exact A and A as the sum of its first T BF16 terms (bf16_split: T = 1 is
  A rounded to BF16; T = 3 is an FP32 A exactly).
* Subsampled randomized Hadamard (Sec. 1.2.1): S = (1/sqrt(d)) P H D with
  m' = 2^ceil(log2 m) (rows m..m'-1 of [A | b] are zero), H the unnormalised
  Sylvester-Hadamard matrix H[p, i] = (-1)^popcount(p & i) applied by the fast
  Walsh-Hadamard transform, D = diag of signs from stream 1, and P the selection
  of d distinct rows of [0, m') drawn by Floyd's algorithm from stream 2, sorted
  ascending.  Reading: sampling without replacement.
"""
import math

import numpy as np
from scipy.special import ndtri

from . import hashing as H

# ---------------------------------------------------------------- CountSketch

def countsketch_matrix(m, d, seed):
    """Dense CountSketch S (d x m, FP64): S[h(i), i] = s(i), zeros elsewhere."""
    h, s = H.countsketch_hash(seed, m, d)
    S = np.zeros((d, m))
    S[h, np.arange(m)] = s
    return S


def countsketch_apply(A, d, seed):
    """SA by the row-scatter form of the definition: SA[k] = sum over rows i with
    h(i) = k of s(i) * A[i].  Works for a matrix or a vector; FP64."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    h, s = H.countsketch_hash(seed, m, d)
    out = np.zeros((d,) + A.shape[1:])
    signed = A * s.reshape((m,) + (1,) * (A.ndim - 1))
    np.add.at(out, h, signed)
    return out


def countsketch_apply_csr(rowptr, col, val, n, d, seed):
    """SA for A given in CSR form (rowptr of length m+1, column indices, values):
    SA[h(i), col] += s(i) * val for every stored entry of row i.  FP64."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    m = len(rowptr) - 1
    h, s = H.countsketch_hash(seed, m, d)
    counts = np.diff(rowptr)
    row_of_entry = np.repeat(np.arange(m), counts)
    out = np.zeros((d, n))
    np.add.at(out, (h[row_of_entry], np.asarray(col, dtype=np.int64)),
              s[row_of_entry] * np.asarray(val, dtype=np.float64))
    return out

# ---------------------------------------------------------------- BF16 helper

def round_to_bf16(x):
    """Round FP64 values to the nearest BF16 number (8 significant bits), ties to
    even, returned as FP64.  Normal range only (the values used here are)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    mant, expo = np.frexp(x[nz])           # x = mant * 2^expo, 0.5 <= |mant| < 1
    scaled = np.ldexp(mant, 8)             # 8 significant bits before the point
    out[nz] = np.ldexp(np.round(scaled), expo - 8)   # np.round: half to even
    return out


def round_to_bf16_via_f32(x):
    """BF16 rounding of FP32 values (round-to-nearest-even on the FP32 bit
    pattern), returned as FP64.  Used for the A operand of the Gaussian path,
    which starts from FP32 data."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_split(x, terms):
    """The first `terms` BF16 terms of FP32 values x (list of FP64 arrays):
    term 1 is x rounded to BF16, term t + 1 is the rounding of the remainder
    x - (term 1 + .. + term t), each remainder computed exactly in FP64."""
    rem = np.asarray(x, dtype=np.float32).astype(np.float64)
    out = []
    for _ in range(terms):
        t = round_to_bf16(rem)
        out.append(t)
        rem = rem - t
    return out


def bf16_terms(x, terms):
    """x as the sum of its first `terms` BF16 terms (FP64)."""
    parts = bf16_split(x, terms)
    total = parts[0].copy()
    for t in parts[1:]:
        total += t
    return total

# ---------------------------------------------------------------- Gaussian

GAUSS_TABLE_BITS = 8


def gaussian_table():
    """T[j] = BF16(Phi^{-1}((j + 1/2) / 256)), j = 0..255, as FP64."""
    n = 1 << GAUSS_TABLE_BITS
    q = ndtri((np.arange(n, dtype=np.float64) + 0.5) / n)
    return round_to_bf16(q)


def gaussian_indices(m, d, seed):
    """Table index j[k, i] (d x m, int64) of every entry of G: byte (i mod 8)
    of output (i div 8) * d + k of stream 3."""
    i = np.arange(m, dtype=np.uint64)[None, :]
    k = np.arange(d, dtype=np.uint64)[:, None]
    counter = (i // np.uint64(8)) * np.uint64(d) + k
    key = H.splitmix64_at(H.stream_state(seed, H.STREAM_GAUSSIAN), counter)
    return ((key >> (np.uint64(8) * (i % np.uint64(8)))) & np.uint64(0xFF)).astype(np.int64)


def gaussian_matrix(m, d, seed):
    """Dense Gaussian sketch S = G / sqrt(d) (d x m, FP64)."""
    return gaussian_table()[gaussian_indices(m, d, seed)] / math.sqrt(d)


def gaussian_apply(A, d, seed, bf16_operand=True, terms=1):
    """SA = (G / sqrt(d)) A.  With bf16_operand the matrix A is first replaced
    by the sum of its first `terms` BF16 terms (the operand the tensor-core path
    multiplies; terms = 1: A rounded to BF16); the product is FP64."""
    A = np.asarray(A)
    Ause = bf16_terms(A, terms) if bf16_operand else A.astype(np.float64)
    S = gaussian_matrix(A.shape[0], d, seed)
    return S @ Ause

# ---------------------------------------------------------------- SRHT

def next_pow2(m):
    return 1 << max(0, (int(m) - 1).bit_length())


def hadamard_matrix(mp):
    """Unnormalised Sylvester-Hadamard matrix of order mp (a power of two):
    H[p, i] = (-1)^popcount(p & i)."""
    p = np.arange(mp)[:, None]
    i = np.arange(mp)[None, :]
    pc = np.vectorize(lambda v: bin(int(v)).count("1"))(p & i)
    return np.where(pc % 2 == 0, 1.0, -1.0)


def fwht(X):
    """Unnormalised fast Walsh-Hadamard transform along axis 0 (length a power of
    two): returns H X, by log2(len) butterfly stages (u, v) -> (u + v, u - v)."""
    X = np.array(X, dtype=np.float64, copy=True)
    n = X.shape[0]
    assert n & (n - 1) == 0
    h = 1
    while h < n:
        Y = X.reshape((n // (2 * h), 2, h) + X.shape[1:])
        u = Y[:, 0].copy()
        v = Y[:, 1].copy()
        Y[:, 0] = u + v
        Y[:, 1] = u - v
        X = Y.reshape(X.shape)
        h *= 2
    return X


def srht_signs(m, seed):
    """Diagonal of D for rows 0..m-1 (float64, +-1), stream 1, bit 63."""
    k = H.splitmix64_at(H.stream_state(seed, H.STREAM_SRHT_SIGN), np.arange(m, dtype=np.uint64))
    return H.sign_of(k)


def srht_sample(mp, d, seed):
    """d distinct row indices of [0, mp), sorted ascending (Floyd's algorithm).

    Step t = 0..d-1 considers the range [0, J], J = mp - d + t, draws
    u = ((k_t mod 2^32) * (J + 1)) >> 32 with k_t output t of stream 2, and keeps u
    unless it was already chosen, in which case it keeps J."""
    assert 1 <= d <= mp < (1 << 32)
    keys = H.splitmix64_at(H.stream_state(seed, H.STREAM_SRHT_SAMPLE), np.arange(d, dtype=np.uint64))
    chosen = set()
    for t in range(d):
        J = mp - d + t
        u = ((int(keys[t]) & 0xFFFFFFFF) * (J + 1)) >> 32
        chosen.add(J if u in chosen else u)
    return np.array(sorted(chosen), dtype=np.int64)


def srht_matrix(m, d, seed):
    """Dense SRHT S = (1/sqrt(d)) P H D restricted to the m real columns (d x m)."""
    mp = next_pow2(m)
    P = srht_sample(mp, d, seed)
    Hm = hadamard_matrix(mp)
    return Hm[P][:, :m] * srht_signs(m, seed)[None, :] / math.sqrt(d)


def srht_apply(A, d, seed):
    """SA by the fast transform: pad [A] to m' rows, multiply by D, FWHT, take the
    sampled rows, scale by 1/sqrt(d)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    mp = next_pow2(m)
    X = np.zeros((mp,) + A.shape[1:])
    X[:m] = A * srht_signs(m, seed).reshape((m,) + (1,) * (A.ndim - 1))
    Y = fwht(X)
    return Y[srht_sample(mp, d, seed)] / math.sqrt(d)

# ---------------------------------------------------------------- dispatch

KINDS = ("countsketch", "gaussian", "srht")


def sketch_apply(kind, A, d, seed, bf16_operand=True, terms=1):
    if kind == "countsketch":
        return countsketch_apply(A, d, seed)
    if kind == "gaussian":
        return gaussian_apply(A, d, seed, bf16_operand=bf16_operand, terms=terms)
    if kind == "srht":
        return srht_apply(A, d, seed)
    raise ValueError(kind)


def sketch_matrix(kind, m, d, seed):
    if kind == "countsketch":
        return countsketch_matrix(m, d, seed)
    if kind == "gaussian":
        return gaussian_matrix(m, d, seed)
    if kind == "srht":
        return srht_matrix(m, d, seed)
    raise ValueError(kind)


def countsketch_rows(A, d, seed, rows):
    """Selected output rows k of SA (and of Sb when A is a vector) straight from
    the definition SA[k] = sum over i with h(i) = k of s(i) A[i]; FP64.  Used to
    check full-size results one output row at a time."""
    A = np.asarray(A)
    m = A.shape[0]
    h, s = H.countsketch_hash(seed, m, d)
    out = []
    for k in rows:
        idx = np.nonzero(h == k)[0]
        out.append((s[idx].reshape((-1,) + (1,) * (A.ndim - 1)) * A[idx].astype(np.float64)).sum(axis=0))
    return np.array(out)


def gaussian_rows(A, d, seed, rows, bf16_operand=True, terms=1):
    """Selected output rows k of (G / sqrt(d)) A (Sec. 1.2.1), each from its own
    row of G: G[k, i] = T[index(k, i)] for all i, then one dot product per
    column; FP64.  Same layout as gaussian_indices, one row at a time, for
    checking full-size results."""
    A = np.asarray(A)
    m = A.shape[0]
    Ause = bf16_terms(A, terms) if bf16_operand else A.astype(np.float64)
    T = gaussian_table()
    i = np.arange(m, dtype=np.uint64)
    state = H.stream_state(seed, H.STREAM_GAUSSIAN)
    out = []
    for k in rows:
        key = H.splitmix64_at(state, (i // np.uint64(8)) * np.uint64(d) + np.uint64(k))
        idx = (key >> (np.uint64(8) * (i % np.uint64(8)))) & np.uint64(0xFF)
        out.append(T[idx.astype(np.int64)] @ Ause / math.sqrt(d))
    return np.array(out)


def _parity(x):
    """Parity of the set bits of each uint64 (XOR folding)."""
    x = x.copy()
    for s in (32, 16, 8, 4, 2, 1):
        x ^= x >> np.uint64(s)
    return x & np.uint64(1)


def srht_rows(A, d, seed, rows):
    """Selected output rows r of the SRHT sketch (Sec. 1.2.1) straight from the
    definition: with p = P[r], row r = (1/sqrt(d)) sum_i (-1)^popcount(p & i)
    D_i A_i over the m real rows (the padding rows are zero); FP64.  For checking
    full-size results one output row at a time."""
    A = np.asarray(A)
    m = A.shape[0]
    P = srht_sample(next_pow2(m), d, seed)
    Ds = srht_signs(m, seed)
    Af = A.astype(np.float64)
    i = np.arange(m, dtype=np.uint64)
    out = []
    for r in rows:
        h = 1.0 - 2.0 * _parity(i & np.uint64(P[r])).astype(np.float64)
        out.append((h * Ds) @ Af / math.sqrt(d))
    return np.array(out)

# ---------------------------------------------------------------- sparse sign

def sparse_sign_hash(m, d, zeta, seed):
    """Rows (m x zeta, int64) and signs (m x zeta, +-1) of the sparse sign
    embedding (Sec. 1.2.2, after Martinsson & Tropp 2020): column i of S holds
    zeta nonzeros +-1/sqrt(zeta) at distinct rows.

    Draw z = 0..zeta-1 of column i uses key k_z: output i of stream 0 for z = 0
    (so zeta = 1 is the CountSketch), output i*(zeta-1) + z-1 of stream 4 for
    z >= 1.  The rows follow Floyd's algorithm on [0, d): draw z considers
    [0, J], J = d - zeta + z, takes u = ((k_z mod 2^32) * (J + 1)) >> 32, and
    keeps u unless an earlier draw of the column took it, in which case it keeps
    J.  The sign of draw z is -1 iff bit 63 of k_z is set."""
    assert 1 <= zeta <= d
    i = np.arange(m, dtype=np.uint64)
    rows = np.zeros((m, zeta), dtype=np.int64)
    signs = np.zeros((m, zeta))
    for z in range(zeta):
        if z == 0:
            k = H.splitmix64_at(H.stream_state(seed, H.STREAM_COUNTSKETCH), i)
        else:
            k = H.splitmix64_at(H.stream_state(seed, H.STREAM_SPARSE_SIGN),
                                i * np.uint64(zeta - 1) + np.uint64(z - 1))
        J = d - zeta + z
        with np.errstate(over="ignore"):
            u = (((k & np.uint64(0xFFFFFFFF)) * np.uint64(J + 1)) >> np.uint64(32)).astype(np.int64)
        taken = np.zeros(m, dtype=bool)
        for zz in range(z):
            taken |= rows[:, zz] == u
        rows[:, z] = np.where(taken, J, u)
        signs[:, z] = H.sign_of(k)
    return rows, signs


def sparse_sign_matrix(m, d, zeta, seed):
    """Dense sparse sign embedding S (d x m, FP64)."""
    rows, signs = sparse_sign_hash(m, d, zeta, seed)
    S = np.zeros((d, m))
    for z in range(zeta):
        S[rows[:, z], np.arange(m)] = signs[:, z] / math.sqrt(zeta)
    return S


def sparse_sign_apply(A, d, zeta, seed):
    """SA by scattering every row into its zeta rows of S (FP64)."""
    A = np.asarray(A, dtype=np.float64)
    rows, signs = sparse_sign_hash(A.shape[0], d, zeta, seed)
    out = np.zeros((d,) + A.shape[1:])
    for z in range(zeta):
        np.add.at(out, rows[:, z], (signs[:, z] / math.sqrt(zeta)).reshape((-1,) + (1,) * (A.ndim - 1)) * A)
    return out
