"""CKKS canonical-embedding encode/decode for the oracle (test infrastructure).

Slots follow the HEAAN convention the paper adopts (Sec. 6: log s slots):
slot j of a plaintext m(X) in Z[X]/(X^N+1) is m(zeta^(5^j mod 2N)) / Delta,
zeta = exp(i pi / N), for j < n = N/2 (full packing).  A message of
n' < N/2 slots is encoded as m(X) = m'(X^(N/(2n'))) with m' the full packing
at ring size 2n' (sparse packing).

The evaluation at all odd powers zeta^(2k+1) is the negacyclic transform of
Sec. 2 (Eq. negacyclic_fft / negacyclic_ifft, with the evaluation point
written as zeta^(+(2k+1))); numpy's FFT serves as the library primitive for
the inner cyclic sum.  Floating point only: not part of the bit-exact
contract.
"""
from __future__ import annotations

import numpy as np


def slot_exponents(N: int, n: int) -> np.ndarray:
    """5^j mod 2N for j < n."""
    out = np.empty(n, dtype=np.int64)
    e = 1
    for j in range(n):
        out[j] = e
        e = e * 5 % (2 * N)
    return out


def evaluate_odd_powers(m, N: int) -> np.ndarray:
    """vals[k] = m(zeta^(2k+1)) for k < N; = sum_j (m_j zeta^j) omega^(jk), omega = zeta^2."""
    m = np.asarray([float(x) for x in m], dtype=np.float64)
    j = np.arange(N)
    tw = np.exp(1j * np.pi * j / N)
    return np.fft.ifft(m * tw) * N


def interpolate_odd_powers(vals: np.ndarray, N: int) -> np.ndarray:
    """Inverse of evaluate_odd_powers: m_j = N^-1 zeta^-j sum_k vals[k] omega^(-jk)."""
    j = np.arange(N)
    return np.fft.fft(vals) / N * np.exp(-1j * np.pi * j / N)


def encode(z, N: int, log_scale: int) -> list[int]:
    """Integer plaintext m with m(zeta^(5^j)) ~= 2^log_scale z_j (rounded to nearest)."""
    z = np.asarray(z, dtype=np.complex128)
    n = z.size
    assert n >= 1 and n <= N // 2 and n & (n - 1) == 0
    Ns = 2 * n  # ring size of the full packing
    vals = np.zeros(Ns, dtype=np.complex128)
    delta = float(2 ** log_scale)
    for jj, e in enumerate(slot_exponents(Ns, n)):
        vals[(e - 1) // 2] = delta * z[jj]
        e2 = 2 * Ns - e  # zeta^-e = conjugate point
        vals[(e2 - 1) // 2] = delta * np.conj(z[jj])
    small = interpolate_odd_powers(vals, Ns).real
    gap = N // Ns
    out = [0] * N
    for i in range(Ns):
        out[i * gap] = int(np.rint(small[i]))
    return out


def decode(m, N: int, log_scale: float, n: int) -> np.ndarray:
    """z_j = m'(zeta'^(5^j)) / 2^log_scale for j < n, m' the lattice part of m.

    m holds centred integers.  As in HEAAN, the coefficients at multiples of
    gap = N/(2n) form m'(Y), Y = X^gap, and the rest (noise only, for a
    sparse packing) is dropped; for n = N/2 this is m itself.
    """
    gap = N // (2 * n)
    Ns = 2 * n
    small = [m[i * gap] for i in range(Ns)]
    vals = evaluate_odd_powers(small, Ns)
    exps = slot_exponents(Ns, n)
    return np.array([vals[(e - 1) // 2] for e in exps]) / float(2.0 ** log_scale)
