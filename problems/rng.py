"""Seeded random numbers for the synthetic Stokes problems.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) produces 64-bit words from a counter; uniforms take
the top 53 bits; normals use the Box-Muller transform.  Every random value the
problems need (vertex perturbations, right-hand sides, batched-instance sizes
and viscosities) is drawn here on the host and stored in the problem, so no
solver component ever draws random numbers.  This module holds no arithmetic
of the solver.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n, offset=0):
    """Return n 64-bit SplitMix64 outputs for counters offset+1 .. offset+n."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, lo=0.0, hi=1.0, offset=0):
    """n uniforms in [lo, hi) from the top 53 bits of SplitMix64 words."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed, n, offset=0):
    """n standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m, offset=offset)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def integers(seed, n, lo, hi, offset=0):
    """n integers uniform on {lo, ..., hi} (inclusive)."""
    u = uniform(seed, n, offset=offset)
    return lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)
