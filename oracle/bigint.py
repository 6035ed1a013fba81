"""Radix-2^32 limb form of big-integer polynomials (Sec. 4, radix representation).

A polynomial with N coefficients of up to 32*L bits is stored as an array of
shape (L, N): limb l of coefficient i at [l, i], least significant limb first
(little-endian limb order), N contiguous.  These are the oracle's own
converters; the CUDA path never calls them.
"""
from __future__ import annotations

import numpy as np


def from_limbs(limbs: np.ndarray, signed: bool = False) -> list[int]:
    """(L, N) uint32 limbs -> list of N Python ints.

    With signed=True the limbs are read as 32*L-bit two's complement.
    """
    limbs = np.ascontiguousarray(np.asarray(limbs, dtype=np.uint32))
    L, N = limbs.shape
    # transpose to coefficient-major, then read each coefficient's bytes
    by = np.ascontiguousarray(limbs.T).astype("<u4").tobytes()
    width = 4 * L
    out = [int.from_bytes(by[i * width:(i + 1) * width], "little") for i in range(N)]
    if signed:
        top = 1 << (32 * L)
        half = top >> 1
        out = [x - top if x >= half else x for x in out]
    return out


def to_limbs(values, L: int) -> np.ndarray:
    """List of N Python ints -> (L, N) uint32 limbs of each value mod 2^(32L).

    Negative values come out in two's complement.
    """
    N = len(values)
    mask = (1 << (32 * L)) - 1
    width = 4 * L
    by = b"".join((int(v) & mask).to_bytes(width, "little") for v in values)
    arr = np.frombuffer(by, dtype="<u4").reshape(N, L)
    return np.ascontiguousarray(arr.T).astype(np.uint32)


def limbs_for_bits(bits: int) -> int:
    return (int(bits) + 31) // 32
