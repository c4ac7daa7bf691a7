"""Pins of the oracle's hash/sign stream (the implicit S of the sketch).

Independent pins: the published SplitMix64 known-answer vector, the integer
range-reduction identity checked with Python big integers, and statistical
uniformity/balance.  The frozen per-seed vectors are a regression pin."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import hashing as H

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t) for t in line.split()])
    return rows


def test_splitmix64_known_answer():
    rows = _read("splitmix64_seed1234567.txt")
    idx = np.array([r[0] for r in rows], dtype=np.uint64)
    got = H.splitmix64_at(np.uint64(1234567), idx)
    assert [int(g) for g in got] == [r[1] for r in rows]


def test_mix64_fixed_point_and_bijective_sample():
    assert int(H.mix64(np.uint64(0))) == 0
    z = np.arange(1, 1 << 16, dtype=np.uint64)
    assert len(np.unique(H.mix64(z))) == z.size      # no collisions on a sample


def test_stream_separation():
    k0 = H.countsketch_keys(5, 32)
    k1 = H.splitmix64_at(H.stream_state(5, 1), np.arange(32, dtype=np.uint64))
    assert not np.any(k0 == k1)
    # stream state is the seed with the stream id in the top byte
    assert int(H.stream_state(5, 3)) == 5 ^ (3 << 56)


@pytest.mark.parametrize("d", [1, 3, 256, 1000, 1024, 2048])
def test_bucket_range_reduction_matches_bigint(d):
    keys = H.countsketch_keys(7, 4096)
    h = H.bucket_of(keys, d)
    ref = [((int(k) & 0xFFFFFFFF) * d) >> 32 for k in keys]
    assert h.tolist() == ref
    assert h.min() >= 0 and h.max() < d


def test_bucket_uniformity_chi2():
    d, m = 1024, 1 << 20
    h, s = H.countsketch_hash(1, m, d)
    counts = np.bincount(h, minlength=d)
    chi2 = ((counts - m / d) ** 2 / (m / d)).sum()
    p = stats.chi2.sf(chi2, d - 1)
    assert 1e-4 < p < 1 - 1e-4
    assert abs(s.sum()) < 5 * np.sqrt(m)            # sign balance


def test_sign_and_bucket_independent():
    d, m = 64, 1 << 18
    h, s = H.countsketch_hash(3, m, d)
    pos = np.bincount(h[s > 0], minlength=d)
    neg = np.bincount(h[s < 0], minlength=d)
    table = np.vstack([pos, neg])
    _, p, _, _ = stats.chi2_contingency(table)
    assert p > 1e-4


@pytest.mark.parametrize("seed", [0, 1])
def test_frozen_countsketch_vectors(seed):
    rows = _read(f"countsketch_hash_seed{seed}.txt")
    k = H.countsketch_keys(seed, 64)
    h = H.bucket_of(k, 1024)
    s = H.sign_of(k)
    assert [int(x) for x in k] == [r[1] for r in rows]
    assert h.tolist() == [r[2] for r in rows]
    assert s.astype(int).tolist() == [r[3] for r in rows]
