"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws random numbers in the shapes and distributions of
the scheme's workloads.  It performs none of the scheme's arithmetic: no
modular reduction, no ring product, no encoding.  Both sides receive the
arrays it returns as plain inputs, so the random values the scheme draws
(secret, error, ephemeral and uniform key polynomials) are identical on
both sides without either side depending on the other.

Distributions (CKKS/HEAAN as adopted by the paper, Sec. 2 and Sec. 6):
  * uniform polynomials mod 2^logQ:   independent uniform 32-bit limbs,
    bits at or above logQ cleared (little-endian limb order, layout
    [..., L, N] with N contiguous);
  * ternary secret / ephemeral poly:  uniform over {-1, 0, 1};
  * sparse ternary secret:            exactly h nonzero coefficients at
    uniformly chosen positions (without replacement), signs uniform;
  * error polynomial:                 rounded normal with sigma = 3.2,
    tails cut at 6 sigma (|e| <= 19);
  * CKKS messages:                    complex numbers uniform in the unit
    disk (rejection sampling);
  * BGV messages:                     integers uniform in [0, t).
"""
from __future__ import annotations

import numpy as np

SIGMA = 3.2
TAIL = 19  # floor(6 * sigma)


def rng(seed: int) -> np.random.Generator:
    """A PCG64 generator; every input of a test or a bench run starts here."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def limb_count(log_bits: int) -> int:
    """Number of 32-bit limbs that hold an unsigned log_bits-bit number."""
    return (int(log_bits) + 31) // 32


def uniform_limbs(g: np.random.Generator, lead_shape, n: int, log_bits: int) -> np.ndarray:
    """Uniform integers in [0, 2^log_bits) as uint32 limbs, shape lead_shape + (L, n)."""
    lead = tuple(lead_shape) if isinstance(lead_shape, (tuple, list)) else (int(lead_shape),)
    L = limb_count(log_bits)
    out = g.integers(0, 1 << 32, size=lead + (L, n), dtype=np.uint64).astype(np.uint32)
    top_bits = log_bits - 32 * (L - 1)
    if top_bits < 32:
        out[..., L - 1, :] &= np.uint32((1 << top_bits) - 1)
    return out


def ternary(g: np.random.Generator, lead_shape, n: int) -> np.ndarray:
    """Uniform {-1, 0, 1} coefficients, int8, shape lead_shape + (n,)."""
    lead = tuple(lead_shape) if isinstance(lead_shape, (tuple, list)) else (int(lead_shape),)
    return (g.integers(0, 3, size=lead + (n,), dtype=np.int64) - 1).astype(np.int8)


def sparse_ternary(g: np.random.Generator, n: int, h: int) -> np.ndarray:
    """Exactly h coefficients in {-1, 1} at distinct uniform positions, int8 (n,)."""
    out = np.zeros(n, dtype=np.int8)
    pos = g.choice(n, size=int(h), replace=False)
    out[pos] = (2 * g.integers(0, 2, size=int(h)) - 1).astype(np.int8)
    return out


def gaussian(g: np.random.Generator, lead_shape, n: int, sigma: float = SIGMA) -> np.ndarray:
    """Rounded normal(0, sigma) coefficients, |e| <= 19, int32, shape lead_shape + (n,)."""
    lead = tuple(lead_shape) if isinstance(lead_shape, (tuple, list)) else (int(lead_shape),)
    e = np.rint(g.normal(0.0, sigma, size=lead + (n,)))
    return np.clip(e, -TAIL, TAIL).astype(np.int32)


def unit_disk(g: np.random.Generator, count: int) -> np.ndarray:
    """count complex numbers uniform in the closed unit disk (rejection sampling)."""
    out = np.empty(0, dtype=np.complex128)
    while out.size < count:
        z = g.uniform(-1.0, 1.0, size=2 * count) + 1j * g.uniform(-1.0, 1.0, size=2 * count)
        out = np.concatenate([out, z[np.abs(z) <= 1.0]])
    return out[:count]


def uniform_mod_t(g: np.random.Generator, lead_shape, n: int, t: int) -> np.ndarray:
    """BGV plaintext coefficients uniform in [0, t), int64, shape lead_shape + (n,)."""
    lead = tuple(lead_shape) if isinstance(lead_shape, (tuple, list)) else (int(lead_shape),)
    return g.integers(0, int(t), size=lead + (n,), dtype=np.int64)


def small_signed(g: np.random.Generator, lead_shape, n: int, log_bound: int) -> np.ndarray:
    """Integers uniform in (-2^log_bound, 2^log_bound), int64 (log_bound <= 62).

    Stands in for the coefficients of an encoded CKKS message at scale
    2^(log_bound - 1) where only the size of the plaintext matters.
    """
    lead = tuple(lead_shape) if isinstance(lead_shape, (tuple, list)) else (int(lead_shape),)
    b = 1 << int(log_bound)
    return g.integers(-b + 1, b, size=lead + (n,), dtype=np.int64)


def poisson_arrivals(g: np.random.Generator, rate_hz: float, duration_s: float) -> np.ndarray:
    """Arrival times of a Poisson process (exponential gaps), seconds."""
    gaps = g.exponential(1.0 / rate_hz, size=int(rate_hz * duration_s * 1.5) + 16)
    t = np.cumsum(gaps)
    return t[t < duration_s]
