"""splitmix64 (Steele, Lea & Flood 2014, constants from Vigna's public-domain
reference) written out for the oracle.  TEST INFRASTRUCTURE ONLY.

The n-th output (n = 1, 2, ...) for seed s is  mix(s + n * 0x9E3779B97F4A7C15)
where mix is the variant-13 finaliser.  The oracle uses it for the tie-break
noise that the method draws inside the similarity build and for the uniform
landmark sample of Algorithm 3 Step 1.
"""
import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MASK = 0xFFFFFFFFFFFFFFFF


def mix(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def output(seed: int, n: int) -> int:
    """The n-th splitmix64 output (1-based) -- plain Python integers."""
    return mix((seed + n * GOLDEN) & MASK)


def outputs(seed: int, ns: np.ndarray) -> np.ndarray:
    """Vectorised ``output`` for an array of 1-based counters (uint64 math)."""
    ns = np.asarray(ns, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK) + ns * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def unit_interval(seed: int, ns: np.ndarray) -> np.ndarray:
    """u in [0,1): top 53 bits of the output times 2^-53."""
    return (outputs(seed, ns) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
