"""Negacyclic ring arithmetic in Z[X]/(X^N + 1) for the oracle (test infrastructure).

Three independent ways to get the exact product over Z:

* ``negacyclic_schoolbook`` -- the definition itself: the full product
  sum_{i,j} a_i b_j X^(i+j) (Sec. 2, Eq. schoolbook) folded with X^N = -1
  (Eq. reduction), in Python integers.  O(N^2); used up to N = 2^11.
* ``negacyclic_kronecker`` -- Kronecker substitution: pack each polynomial
  into one big integer at X = 2^w, multiply with Python's integer product,
  unpack the 2N - 1 balanced digits and fold.  Used up to N = 2^12.
* ``negacyclic_fast`` -- the C routine in fastmul.c (62-bit-prime NTTs and a
  full multi-precision CRT), for large N.

``negacyclic_mul`` picks one by size.  All three return exact integers; the
callers reduce modulo Q themselves.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import bigint

_HERE = os.path.dirname(os.path.abspath(__file__))
_FAST_SO = os.path.join(_HERE, "_fastmul.so")


def build_fast(force: bool = False) -> str:
    """Compile fastmul.c into _fastmul.so (plain gcc, no CPU-specific flags)."""
    src = os.path.join(_HERE, "fastmul.c")
    if force or not os.path.exists(_FAST_SO) or os.path.getmtime(_FAST_SO) < os.path.getmtime(src):
        import subprocess

        tmp = _FAST_SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _FAST_SO)
    return _FAST_SO


_lib = None


def _fast_lib():
    global _lib
    if _lib is None:
        build_fast()
        lib = ctypes.CDLL(_FAST_SO)
        lib.oracle_negacyclic_mul.restype = ctypes.c_int
        lib.oracle_negacyclic_mul.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        _lib = lib
    return _lib


def _max_bits(v) -> int:
    return max((abs(int(x)).bit_length() for x in v), default=0)


def negacyclic_schoolbook(a, b) -> list[int]:
    """Exact c = a*b in Z[X]/(X^N+1) by Eq. schoolbook then Eq. reduction (Sec. 2)."""
    N = len(a)
    assert len(b) == N
    full = [0] * (2 * N)
    for i in range(N):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(N):
            full[i + j] += ai * int(b[j])
    return [full[i] - full[N + i] for i in range(N)]


def negacyclic_kronecker(a, b) -> list[int]:
    """Exact negacyclic product by Kronecker substitution in Python integers."""
    N = len(a)
    assert len(b) == N
    bound_bits = _max_bits(a) + _max_bits(b) + N.bit_length() + 2
    w = ((bound_bits + 7) // 8) * 8  # digit width in bits, whole bytes
    A = 0
    B = 0
    for i in reversed(range(N)):
        A = (A << w) + int(a[i])
        B = (B << w) + int(b[i])
    C = A * B
    # offset every digit by 2^(w-1) so all digits are non-negative, then slice bytes
    ndig = 2 * N - 1
    offset = sum(1 << (w * k + w - 1) for k in range(ndig))
    C += offset
    nbytes = w // 8
    by = C.to_bytes(nbytes * ndig + 1, "little")
    half = 1 << (w - 1)
    full = [int.from_bytes(by[k * nbytes:(k + 1) * nbytes], "little") - half for k in range(ndig)] + [0]
    return [full[i] - full[N + i] for i in range(N)]


def negacyclic_fast(a, b, out_bits: int | None = None) -> list[int]:
    """Exact negacyclic product via the C oracle (fastmul.c)."""
    N = len(a)
    assert len(b) == N and N & (N - 1) == 0
    logN = N.bit_length() - 1
    ba, bb = _max_bits(a), _max_bits(b)
    La = ba // 32 + 1  # room for a sign bit
    Lb = bb // 32 + 1
    bound = ba + bb + logN
    Lout = (bound + 1) // 32 + 1 if out_bits is None else (out_bits + 31) // 32
    la = bigint.to_limbs(a, La)
    lb = bigint.to_limbs(b, Lb)
    out = np.zeros((Lout, N), dtype=np.uint32)
    rc = _fast_lib().oracle_negacyclic_mul(logN, la.ctypes.data, La, 1, lb.ctypes.data, Lb, 1, out.ctypes.data,
                                           Lout, bound)
    if rc != 0:
        raise RuntimeError(f"oracle_negacyclic_mul failed: {rc}")
    return bigint.from_limbs(out, signed=True)


def negacyclic_mul(a, b) -> list[int]:
    """Exact negacyclic product; picks the plain method the size allows."""
    N = len(a)
    if N <= 64:
        return negacyclic_schoolbook(a, b)
    if N <= 512:
        return negacyclic_kronecker(a, b)
    return negacyclic_fast(a, b)


def mod_poly(a, m: int) -> list[int]:
    """Coefficient-wise canonical residue in [0, m)."""
    return [int(x) % m for x in a]


def add_poly(a, b) -> list[int]:
    return [int(x) + int(y) for x, y in zip(a, b)]


def sub_poly(a, b) -> list[int]:
    return [int(x) - int(y) for x, y in zip(a, b)]


def scale_poly(a, c: int) -> list[int]:
    return [int(x) * c for x in a]


def automorphism(a, g: int) -> list[int]:
    """kappa_g: a(X) -> a(X^g) in Z[X]/(X^N+1), g odd (Sec. 2, Galois automorphisms).

    X^i maps to X^(i g mod 2N); an exponent e >= N is X^(e-N) * X^N = -X^(e-N).
    """
    N = len(a)
    assert g % 2 == 1
    out = [0] * N
    for i in range(N):
        e = (i * g) % (2 * N)
        if e < N:
            out[e] += int(a[i])
        else:
            out[e - N] -= int(a[i])
    return out
