"""Known-answer pins of the oracle's point streams (reading R1 of Sec. 3.2's seeded sampling).

Point i of hash k is output i+1 of a SplitMix64 generator whose state starts at
s_k, and s_k is output k+1 of a SplitMix64 generator whose state starts at the
global seed.  Two independent checks, neither of which reuses the oracle's code:

* the published first outputs of SplitMix64 seeded with 0
  (tests/golden/splitmix64_seed0.txt) fix the generator itself: a wrong shift,
  multiplier or gamma in the oracle's mixer changes them;
* a sequential SplitMix64 written here from the published description (the
  state advances by the golden gamma and is then mixed), itself checked against
  those outputs, fixes how streams and points are derived from it, on seeds and
  indices whose state additions wrap past 2^64.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
MASK = (1 << 64) - 1


class SplitMix64:
    """Sequential SplitMix64: the state advances by gamma, each output is the state mixed
    by two xor-shift-multiply rounds and a final xor-shift."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, state: int):
        self.state = state & MASK

    def next(self) -> int:
        self.state = (self.state + self.GAMMA) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def nth(self, n: int) -> int:
        """Output n (1-based) of a fresh copy of this generator."""
        g = SplitMix64(self.state)
        v = 0
        for _ in range(n):
            v = g.next()
        return v


def published():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            idx, val = line.split()
            out.append((int(idx), int(val, 16)))
    return out


def test_published_vectors_fix_the_independent_generator():
    g = SplitMix64(0)
    for idx, val in published():
        assert g.next() == val, idx


def test_oracle_mixer_reproduces_published_vectors(orc):
    # output n of the generator seeded with 0 is mix64(n * gamma)
    for idx, val in published():
        assert orc.mix64((idx * SplitMix64.GAMMA) & MASK) == val, idx


def test_oracle_stream_seeds_are_splitmix_outputs_of_the_global_seed(orc):
    # seed 0: s_k is the published output k + 1
    for idx, val in published():
        assert orc.stream_seed(0, idx - 1) == val
    rng = np.random.default_rng(5)
    seeds = [0x5EED, MASK, MASK - 0x9E3779B97F4A7C15 + 3, 1 << 63] + \
        [int(s) for s in rng.integers(0, 1 << 63, 4, dtype=np.uint64)]
    for seed in seeds:
        for k in (0, 1, 2, 31, 127, 255, 4095):
            assert orc.stream_seed(seed, k) == SplitMix64(seed).nth(k + 1), (seed, k)


def test_oracle_stream_points_follow_the_reading(orc):
    rng = np.random.default_rng(9)
    seeds = [0x5EED, MASK, 1 << 63] + [int(s) for s in rng.integers(0, 1 << 63, 3, dtype=np.uint64)]
    for seed in seeds:
        for k in (0, 5, 127):
            sk = SplitMix64(seed).nth(k + 1)
            g = SplitMix64(sk)
            seq = [g.next() for _ in range(300)]
            for i in (0, 1, 2, 99, 299):
                assert orc.stream_value(seed, k, i) == seq[i], (seed, k, i)
            # x = low 16 bits, y = the next 16 bits
            x, y = orc.stream_points(seed, k, 0, 300)
            assert np.array_equal(x.astype(np.int64), np.array([v & 0xFFFF for v in seq]))
            assert np.array_equal(y.astype(np.int64), np.array([(v >> 16) & 0xFFFF for v in seq]))
    # far indices: output i + 1 of stream k is mix64(s_k + (i + 1) * gamma) with wrap-around;
    # checked by stepping the independent generator's state directly
    for seed, k, i in ((0x5EED, 3, 1 << 20), (MASK, 200, (1 << 24) - 1), (12345, 0, 987654)):
        sk = SplitMix64(seed).nth(k + 1)
        g = SplitMix64((sk + i * SplitMix64.GAMMA) & MASK)
        assert orc.stream_value(seed, k, i) == g.next()
