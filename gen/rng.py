"""Counter-based random stream for the synthetic workloads.

Every workload in this repository is drawn from one generator: the SplitMix64
sequence of Steele, Lea and Flood ("Fast splittable pseudorandom number
generators", OOPSLA 2014), evaluated by counter so that a block of draws is one
vectorised numpy expression.  Only integer arithmetic decides a value; floats
appear only after the 64-bit word is fixed, and every probability table is
quantised to 32-bit integer thresholds before it is compared with a draw, so
x86 and Arm hosts (and any numpy version) produce the same graphs.

This module holds no part of the enumeration method.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function, applied elementwise to uint64 words."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sub_seed(master: int, index: int) -> int:
    """Deterministic child seed number `index` of `master`."""
    x = np.array([(master + (index + 1) * 0xD1B54A32D192ED03) & _MASK64], dtype=np.uint64)
    return int(_mix(x)[0])


class Stream:
    """A SplitMix64 stream: draw i is mix(seed + (i + 1) * gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & _MASK64)
        self.pos = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + 1 + count, dtype=np.uint64)
        self.pos += count
        with np.errstate(over="ignore"):
            return _mix(self.seed + idx * _GAMMA)

    def u32(self, count: int) -> np.ndarray:
        return (self.u64(count) >> np.uint64(32)).astype(np.uint32)

    def below(self, bound: int, count: int) -> np.ndarray:
        """Integers in [0, bound) by the multiply-shift map of a 32-bit draw."""
        if bound <= 0:
            raise ValueError("bound must be positive")
        if bound >= 1 << 32:
            raise ValueError("bound must fit in 32 bits")
        u = self.u32(count).astype(np.uint64)
        return ((u * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)

    def one_below(self, bound: int) -> int:
        return int(self.below(bound, 1)[0])

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits of each draw."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def choice_thresholds(self, thresholds: np.ndarray, count: int) -> np.ndarray:
        """Category index for each draw, given cumulative uint32 thresholds.

        thresholds[i] is the quantised cumulative probability of categories
        0..i (the last entry is 2**32 - 1 or larger); category i is chosen when
        the draw is below thresholds[i] and not below thresholds[i - 1].
        """
        u = self.u32(count).astype(np.uint64)
        return np.searchsorted(thresholds.astype(np.uint64), u, side="right").astype(np.int64)


def quantise_cdf(weights) -> np.ndarray:
    """Cumulative 32-bit thresholds of a discrete distribution.

    The weights are first rounded to integers on a 2**40 scale, so the
    thresholds depend only on exactly rounded float operations.
    """
    w = np.asarray(weights, dtype=np.float64)
    if np.any(w < 0) or w.sum() <= 0:
        raise ValueError("weights must be non-negative with a positive sum")
    wi = np.floor(w / w.max() * float(1 << 40) + 0.5).astype(np.int64)
    cum = np.cumsum(wi, dtype=np.int64)
    total = int(cum[-1])
    # floor(cum * 2^32 / total) in exact integer arithmetic
    thr = np.array([(int(c) << 32) // total for c in cum], dtype=np.uint64)
    thr[-1] = np.uint64((1 << 32))
    return thr
