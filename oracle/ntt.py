"""NTT-friendly primes and the negacyclic NTT as literal sums (test infrastructure).

The transforms here are the O(N^2) direct sums of Sec. 2:

  Eq. negacyclic_ntt:   abar_i = sum_j a_j psi^((2i+1) j)            (mod q)
  Eq. negacyclic_intt:  a_i    = N^-1 psi^-i sum_j abar_j omega^(-ij) (mod q)

with omega = psi^2 and psi a primitive 2N-th root of unity, q = 1 (mod 2N).
They exist to pin the pointwise-product identity of Eq. ntt_mul against the
schoolbook product on small N; the product path never sees these values
(its transform-domain order is internal).
"""
from __future__ import annotations


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases up to 37)."""
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(count: int, two_n: int, lo_bits: int = 30, hi_bits: int = 31) -> list[int]:
    """`count` primes q = 1 (mod two_n) in (2^lo_bits, 2^hi_bits), largest first (Sec. 4)."""
    out = []
    q = ((1 << hi_bits) - 1) // two_n * two_n + 1
    while len(out) < count:
        if q <= (1 << lo_bits):
            raise ValueError("not enough primes in range")
        if is_prime(q):
            out.append(q)
        q -= two_n
    return out


def primitive_2n_root(q: int, N: int) -> int:
    """Smallest psi with psi^N = -1 (mod q), i.e. of order exactly 2N (N a power of two)."""
    assert (q - 1) % (2 * N) == 0
    for x in range(2, q):
        psi = pow(x, (q - 1) // (2 * N), q)
        if pow(psi, N, q) == q - 1:
            return psi
    raise ValueError("no root")


def ntt_direct(a, q: int, psi: int) -> list[int]:
    """Eq. negacyclic_ntt by its definition: abar_i = sum_j a_j psi^((2i+1)j) mod q."""
    N = len(a)
    return [sum(int(a[j]) * pow(psi, (2 * i + 1) * j, q) for j in range(N)) % q for i in range(N)]


def intt_direct(abar, q: int, psi: int) -> list[int]:
    """Eq. negacyclic_intt by its definition: a_i = N^-1 psi^-i sum_j abar_j omega^-ij mod q."""
    N = len(abar)
    omega_inv = pow(psi * psi % q, q - 2, q)
    n_inv = pow(N, q - 2, q)
    psi_inv = pow(psi, q - 2, q)
    out = []
    for i in range(N):
        s = sum(int(abar[j]) * pow(omega_inv, i * j, q) for j in range(N)) % q
        out.append(n_inv * pow(psi_inv, i, q) % q * s % q)
    return out


def ntt_mul_mod_q(a, b, q: int, psi: int) -> list[int]:
    """Eq. ntt_mul: c = iNTT(NTT(a) (.) NTT(b)) mod q, through the direct sums."""
    A = ntt_direct(a, q, psi)
    B = ntt_direct(b, q, psi)
    return intt_direct([x * y % q for x, y in zip(A, B)], q, psi)
