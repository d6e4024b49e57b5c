"""SplitMix64 counter-based generator (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written from its published
definition: out(x) = mix(x + 0x9E3779B97F4A7C15) with the 64-bit finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.

The AMG aggregation draws its node priorities and the power-iteration start
vector from this counter-based stream, so that the same numbers can be
regenerated independently anywhere from (counter) alone.  Oracle copy: test
infrastructure only.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x) -> np.ndarray:
    """SplitMix64 output for counter value(s) x (uint64, wrapping arithmetic)."""
    z = np.asarray(x, dtype=np.uint64) + _GAMMA
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def node_priority(n: int, level: int) -> np.ndarray:
    """32-bit aggregation priority of nodes 0..n-1 on a given AMG level:
    the high 32 bits of splitmix64(i + level * 2^32)."""
    i = np.arange(n, dtype=np.uint64) + (np.uint64(level) << np.uint64(32))
    return (splitmix64(i) >> np.uint64(32)).astype(np.int64)


def unit_uniform(n: int, stream: int) -> np.ndarray:
    """u_i = (splitmix64(i + stream * 2^32) >> 11) * 2^-53 in [0, 1)."""
    i = np.arange(n, dtype=np.uint64) + (np.uint64(stream) << np.uint64(32))
    return (splitmix64(i) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
