"""Counter-based random numbers for the oracle (test infrastructure only).

The eigensolver draws random vectors in two places: the start vector of an
eigenpair extension (Algorithm 4, first step) and the replacement vector after
a Lanczos breakdown (Algorithm 3, the beta < eps branch).  Both the oracle and
the CUDA library draw them from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) used as a counter
generator: entry i of stream s under seed S is

    key  = mix(S + (s + 1) * GAMMA)
    bits = mix(key + (i + 1) * GAMMA)
    x_i  = 2 * (bits >> 11) * 2^-53 - 1            in [-1, 1)

where GAMMA = 0x9E3779B97F4A7C15 and mix is the SplitMix64 finaliser.
This file is an independent implementation of that published definition.
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


def uniform_pm1(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [-1, 1) from stream ``stream`` of ``seed``."""
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream + 1) * GAMMA)
        idx = np.arange(1, n + 1, dtype=np.uint64)
        bits = _mix(key + idx * GAMMA)
    return 2.0 * (bits >> np.uint64(11)).astype(np.float64) * (2.0**-53) - 1.0
