"""Counter-based splitmix64 stream used by the RANDOM bytecode.

Test infrastructure only (see the package docstring).

splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; Vigna's public-domain C version) advances a
64-bit state by the odd constant GAMMA and returns a mixed copy of it: the
k-th output (k = 0, 1, ...) of the generator seeded with ``s`` is
``mix(s + (k + 1) * GAMMA)``. The RANDOM bytecode evaluates that formula at
the counter ``c = key + step * m`` for element ``m``, and maps the output
to [0, 1) by its top 53 bits: ``(z >> 11) * 2^-53`` (exact in float64).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1


def mix64(z: np.ndarray) -> np.ndarray:
    """The splitmix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def counter_state(seed: int, key: int, step: int, m: np.ndarray) -> np.ndarray:
    """``seed + (key + step*m + 1) * GAMMA`` modulo 2^64."""
    m = np.asarray(m, dtype=np.uint64)
    c = np.uint64(key & MASK) + np.uint64(step & MASK) * m
    return np.uint64(seed & MASK) + (c + np.uint64(1)) * np.uint64(GAMMA)


def random_u01(seed: int, key: int, step: int, m: np.ndarray) -> np.ndarray:
    """float64 uniforms in [0, 1) for element indices ``m``."""
    with np.errstate(over="ignore"):
        z = mix64(counter_state(seed, key, step, m))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
