"""Counter-based SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; the 64-bit finaliser with the constants of
Vigna's public-domain reference).

Element i of the stream for a 64-bit key is mix(key + (i + 1) * GAMMA): the
same numbers as the sequential generator started at state = key, but any
element can be drawn on its own, so arrays are filled in one vectorised call
and the result does not depend on the platform or on numpy's own generators.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def derive_key(*parts):
    """Fold integers into one 64-bit key (each part passed through the mixer)."""
    key = np.uint64(0x243F6A8885A308D3)
    for p in parts:
        with np.errstate(over="ignore"):
            key = _mix(np.array([key ^ np.uint64(int(p) & 0xFFFFFFFFFFFFFFFF)],
                                dtype=np.uint64))[0]
            key = np.uint64(key + GAMMA)
    return np.uint64(key)


def splitmix64_stream(key, count, start=0):
    """uint64 array: elements start .. start+count-1 of the stream for `key`."""
    i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(key) + i * GAMMA
    return _mix(state)


def uniform01(key, count, start=0):
    """Doubles in [0, 1) from the top 53 bits of each stream element."""
    bits = splitmix64_stream(key, count, start) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def standard_normal(key, count):
    """Standard normal draws by the Box-Muller transform on stream pairs."""
    m = (count + 1) // 2
    u = uniform01(key, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]
