"""Counter-based Rademacher draws for the stochastic orbitals theta^xi (Sec. II).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper draws theta^xi_Q = +-1 at random (the definition above Eq. 9) and
needs two independent sets, theta and theta' (Eq. 25).  To make the draws
reproducible on two independent implementations, each element is a pure
function of (seed, set, xi, Q):

    counter = set * 2^60 + xi * 2^20 + Q          (xi < 2^40, Q < 2^20)
    z       = first output of SplitMix64 started from state (seed XOR counter)
    theta   = -1 if bit 63 of z is set else +1

SplitMix64 is the generator of Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014: the state advances by the odd
constant 0x9E3779B97F4A7C15 and each output is the advanced state passed
through two xor-shift-multiply rounds and a final xor-shift (shifts 30, 27,
31; multipliers 0xBF58476D1CE4E5B9 and 0x94D049BB133111EB).
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _mix_int(z: int) -> int:
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def splitmix64_stream(state: int, count: int) -> list[int]:
    """The first `count` outputs of SplitMix64 from `state` (Python ints)."""
    out = []
    for _ in range(count):
        state = (state + _GOLDEN) & _MASK
        out.append(_mix_int(state))
    return out


def splitmix64_first(states: np.ndarray) -> np.ndarray:
    """Vectorised first output of SplitMix64 for an array of uint64 states."""
    z = np.asarray(states, dtype=np.uint64) + np.uint64(_GOLDEN)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def rademacher(seed: int, set_index: int, n_s: int, n_aux: int,
               xi_offset: int = 0) -> np.ndarray:
    """theta[xi, Q] in {-1, +1} as float64, shape [n_s, n_aux]."""
    if n_aux >= (1 << 20) or xi_offset + n_s >= (1 << 40) or set_index not in (0, 1):
        raise ValueError("counter field overflow")
    xi = np.arange(xi_offset, xi_offset + n_s, dtype=np.uint64)[:, None]
    q = np.arange(n_aux, dtype=np.uint64)[None, :]
    counter = (np.uint64(set_index) << np.uint64(60)) | (xi << np.uint64(20)) | q
    z = splitmix64_first(np.uint64(seed & _MASK) ^ counter)
    return 1.0 - 2.0 * (z >> np.uint64(63)).astype(np.float64)
