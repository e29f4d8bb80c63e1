"""Counter-based SplitMix64 stream -> U[0,1) doubles.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output of a stream seeded with `s` is
mix(s + (i+1)*GAMMA) with GAMMA = 0x9E3779B97F4A7C15 and the published
finaliser mix().  A double in [0,1) takes the top 53 bits.

The stream is counter-based, so the same (seed, index) gives the same number
on any machine; every synthetic input in `scenes` is drawn from it.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential view of the counter-based stream for one seed."""

    def __init__(self, seed):
        self.seed = np.uint64(seed)
        self.count = 0

    def bits(self, n):
        idx = np.arange(self.count + 1, self.count + n + 1, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            return _mix(self.seed + idx * _GAMMA)

    def uniform(self, n, lo=0.0, hi=1.0):
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u
