"""Writes tests/golden/countsketch_hash_seed{0,1}.txt: the first 64 CountSketch keys,
buckets (d = 1024) and signs of seeds 0 and 1.  Calls only the oracle, so the
frozen values are a regression pin of the oracle's hash stream (its independent
pin is the SplitMix64 known-answer file)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import hashing  # noqa: E402


def main():
    for seed in (0, 1):
        k = hashing.countsketch_keys(seed, 64)
        h = hashing.bucket_of(k, 1024)
        s = hashing.sign_of(k)
        with open(os.path.join(HERE, f"countsketch_hash_seed{seed}.txt"), "w") as f:
            f.write(f"# CountSketch stream (stream 0) of seed {seed}: row, key, bucket (d=1024), sign\n")
            f.write("# written by tests/golden/make_hash_vectors.py from the oracle\n")
            for i in range(64):
                f.write(f"{i} {int(k[i])} {int(h[i])} {int(s[i])}\n")


if __name__ == "__main__":
    main()
