"""Counter-based SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014).

Every synthetic input of this repository is drawn from here, so that the CPU
oracle and the CUDA path see byte-identical inputs.  The generator is written
from its published definition: the state advances by the golden-ratio
increment 0x9E3779B97F4A7C15 and each output is the state passed through the
two xor-shift-multiply finalisation rounds (multipliers 0xBF58476D1CE4E5B9 and
0x94D049BB133111EB, shifts 30/27/31).  Here the state of draw ``i`` of a
stream is ``seed + (i + 1) * increment`` (counter form), which lets numpy draw
whole arrays at once.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """One independent stream of 64-bit draws: ``Stream(seed, tag)``.

    ``tag`` is a small integer naming the purpose of the draws (rate factors,
    temperatures, ...); streams with different tags are decorrelated by
    passing ``seed`` and ``tag`` through the finaliser before use.
    """

    def __init__(self, seed, tag=0):
        with np.errstate(over="ignore"):
            s = _mix(np.uint64(seed) * _GOLDEN + np.uint64(tag))
            self._base = _mix(s ^ np.uint64(0xD1B54A32D192ED03))
        self._next = 0

    def skip(self, n):
        """Advance past n draws (the stream of a batch that starts at a later
        cell); returns self."""
        self._next += int(n)
        return self

    def u64(self, n):
        i = np.arange(self._next, self._next + n, dtype=np.uint64)
        self._next += n
        with np.errstate(over="ignore"):
            return _mix(self._base + (i + np.uint64(1)) * _GOLDEN)

    def uniform(self, n, lo=0.0, hi=1.0):
        """Doubles in [lo, hi): the top 53 bits of each draw times 2**-53."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def uniform_open(self, n):
        """Doubles in (0, 1): top 53 bits plus one half ulp (no zero)."""
        return ((self.u64(n) >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)

    def integers(self, n, k):
        """Integers in [0, k) by multiply-shift of the top 32 bits."""
        hi = (self.u64(n) >> np.uint64(32)).astype(np.uint64)
        with np.errstate(over="ignore"):
            return ((hi * np.uint64(k)) >> np.uint64(32)).astype(np.int64)

    def normal(self, n):
        """Standard normals by the Box-Muller transform; normal i uses draws
        2i and 2i+1, so a prefix of a longer request is unchanged."""
        z = self.u64(2 * n) >> np.uint64(11)
        u1 = (z[0::2].astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
        u2 = z[1::2].astype(np.float64) * (1.0 / 9007199254740992.0)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def log_uniform(self, n, lo, hi):
        return np.exp(self.uniform(n, np.log(lo), np.log(hi)))
