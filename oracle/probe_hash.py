"""Counter-based Rademacher probes for the diagonal estimator (oracle side).

Sec. 3.1 draws each probe component from the Rademacher distribution and
Algorithm 1 draws a fresh set p_1..p_K every EM iteration.  So that the CPU
oracle and the GPU path see the same probes without storing them, each sign
is a pure function of (seed, t, k, d), built from the SplitMix64 output
function (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the 64-bit finaliser with the constants of
Stafford's "Mix13"):

    mix64(x):  z = x + 0x9E3779B97F4A7C15
               z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
               z = (z ^ (z >> 27)) * 0x94D049BB133111EB
               return z ^ (z >> 31)                      (all mod 2^64)

Key schedule (a reading: the paper does not say how probes are drawn):

    s0 = mix64(seed)
    s1 = mix64(s0 ^ t)                 t = 1-based EM iteration number
    h  = mix64(s1 ^ ((d << 8) | w))    d = coordinate, w = k // 64 (< 256)
    p_kd = +1 if bit (k mod 64) of h is 0, else -1

Pins: the raw SplitMix64 stream against its published first outputs, and the
sign statistics (mean, pairwise correlation, bit balance) in the tests.
"""
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1
MAX_K = 64 * 256


def mix64_int(x: int) -> int:
    """SplitMix64 output function on one Python int (mod 2^64)."""
    z = (x + GAMMA) & MASK
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def mix64(x: np.ndarray) -> np.ndarray:
    """Same function, elementwise on a uint64 array (numpy wraps mod 2^64)."""
    z = np.asarray(x, dtype=np.uint64) + np.uint64(GAMMA)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
    return z ^ (z >> np.uint64(31))


def iteration_key(seed: int, t: int) -> int:
    """s1 = mix64(mix64(seed) ^ t)."""
    return mix64_int(mix64_int(seed & MASK) ^ (t & MASK))


def probe_words(seed: int, t: int, D: int, n_words: int) -> np.ndarray:
    """h[d, w] for d < D, w < n_words (uint64, shape D x n_words)."""
    if n_words > 256:
        raise ValueError("at most 256 words (K <= 16384)")
    s1 = np.uint64(iteration_key(seed, t))
    d = np.arange(D, dtype=np.uint64)[:, None]
    w = np.arange(n_words, dtype=np.uint64)[None, :]
    return mix64(s1 ^ ((d << np.uint64(8)) | w))


def probe_matrix(seed: int, t: int, K: int, D: int) -> np.ndarray:
    """Probe block P (D x K, float64 entries +-1), column k = p_{k+1}."""
    if K < 1 or K > MAX_K:
        raise ValueError("K out of range")
    n_words = (K + 63) // 64
    h = probe_words(seed, t, D, n_words)
    k = np.arange(K)
    bits = (h[:, k // 64] >> (k % 64).astype(np.uint64)) & np.uint64(1)
    return 1.0 - 2.0 * bits.astype(np.float64)
