"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers only; it holds none of the method's
arithmetic.  Both the CUDA path and the oracle receive what it returns.

RTGV parameters (Sec. "Randomized Taylor-Green vortex flow", Eq. (initialRTGV)):
24 iid X ~ U[-w, w] per sample, w = 0.025.  The draw is Philox4x64-10
(Salmon et al., SC'11) keyed by (seed, 0); the 24 values of sample m are the
outputs of counters (b, m, 0, 0), b = 0..5, four 64-bit words each, mapped by
U = (x >> 11) 2^-53 and X = w (2U - 1).  numpy's Philox increments its counter
before each block, so starting it at (b, m) - 1 reproduces that stream.
"""
import numpy as np

RTGV_WIDTH = 0.025
_ONES = np.uint64(0xFFFFFFFFFFFFFFFF)


def philox_counter_before(block, m):
    """The numpy Philox counter that yields counter (block, m, 0, 0) on its next block."""
    c = np.array([block, m, 0, 0], dtype=np.uint64)
    # subtract one with borrow across the 256-bit counter
    for k in range(4):
        if c[k] != 0:
            c[k] -= np.uint64(1)
            break
        c[k] = _ONES
    return c


def draw_params(seed, M, w=RTGV_WIDTH, first_sample=0):
    """[M][24] float64 RTGV parameters of samples first_sample .. first_sample+M-1."""
    out = np.empty((M, 24), dtype=np.float64)
    for j in range(M):
        m = first_sample + j
        bg = np.random.Philox(key=np.uint64(seed), counter=philox_counter_before(0, m))
        raw = bg.random_raw(24).astype(np.uint64)
        U = (raw >> np.uint64(11)).astype(np.float64) * 2.0**-53
        out[j] = w * (2.0 * U - 1.0)
    return out


def uniform(seed, shape, low=-1.0, high=1.0):
    """Seeded uniform numbers (test perturbations, random node states)."""
    return np.random.default_rng(seed).uniform(low, high, size=shape)


def normal(seed, shape, scale=1.0):
    """Seeded normal numbers (test perturbations)."""
    return np.random.default_rng(seed).normal(0.0, scale, size=shape)
