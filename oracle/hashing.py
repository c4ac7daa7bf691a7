"""Counter-based random streams that define the implicit sketch S (step "generate S",
Sec. 1.2 of the paper).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper describes the Clarkson-Woodruff sketch only as sparse with random
signs (Sec. 1.2.2); it fixes no generator.  Reading used
here (shared, as a specification only, with the CUDA library, which implements
it separately):

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): a state advanced by the odd constant
  gamma = 0x9E3779B97F4A7C15, each output passed through the "mix64" finaliser
  (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
  0x94D049BB133111EB, xor-shift 31).  Output number i (0-based) of a generator
  seeded with state s0 is mix64(s0 + (i + 1) * gamma), so any output can be
  computed directly from its index (counter-based).
* Stream separation: s0 = seed XOR (stream << 56), with stream 0 = CountSketch,
  1 = SRHT signs, 2 = SRHT row sampling, 3 = Gaussian entries, 4 = the extra
  draws of the sparse sign embedding.
* Bucket of row i:  h(i) = ((k mod 2^32) * d) >> 32  (multiply-shift range
  reduction, Lemire 2019), k = output i of stream 0.
* Sign of row i:  s(i) = -1 if bit 63 of k is set, else +1.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MUL1 = np.uint64(0xBF58476D1CE4E5B9)
MUL2 = np.uint64(0x94D049BB133111EB)

STREAM_COUNTSKETCH = 0
STREAM_SRHT_SIGN = 1
STREAM_SRHT_SAMPLE = 2
STREAM_GAUSSIAN = 3
STREAM_SPARSE_SIGN = 4


def mix64(z):
    """SplitMix64 output finaliser on a uint64 array (arithmetic mod 2^64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * MUL1
        z = (z ^ (z >> np.uint64(27))) * MUL2
    return z ^ (z >> np.uint64(31))


def stream_state(seed, stream):
    """Initial SplitMix64 state of stream `stream` for user seed `seed`."""
    return np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) << np.uint64(56))


def splitmix64_at(state0, idx):
    """Output number `idx` (0-based, uint64 array) of SplitMix64 seeded with `state0`."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state0) + (idx + np.uint64(1)) * GAMMA
    return mix64(z)


def countsketch_keys(seed, m, start=0):
    """Raw 64-bit keys k(i) of CountSketch rows start..start+m-1."""
    idx = np.arange(start, start + m, dtype=np.uint64)
    return splitmix64_at(stream_state(seed, STREAM_COUNTSKETCH), idx)


def bucket_of(keys, d):
    """h(i) = ((k mod 2^32) * d) >> 32, an integer in [0, d)."""
    lo = keys & np.uint64(0xFFFFFFFF)
    with np.errstate(over="ignore"):
        return ((lo * np.uint64(d)) >> np.uint64(32)).astype(np.int64)


def sign_of(keys):
    """s(i) = -1 if bit 63 of the key is set, +1 otherwise (as float64)."""
    return np.where((keys >> np.uint64(63)) == np.uint64(1), -1.0, 1.0)


def countsketch_hash(seed, m, d):
    """Bucket ids h (int64, in [0, d)) and signs s (float64, +-1) of rows 0..m-1."""
    k = countsketch_keys(seed, m)
    return bucket_of(k, d), sign_of(k)
