"""Integer CRT, Garner's mixed-radix conversion, centred reduction (test infrastructure).

  RNS decomposition (Sec. 2):          x_i = X mod q_i
  CRT composition, Eq. crt_composition: X = | sum_i x_i qhat_i [qhat_i^-1]_{q_i} |_Q
  Garner / MRC, Eq. garner_mrc:        X = v_0 + v_1 q_0 + ... + v_{r-1} prod_{i<r-1} q_i,
                                        v_k from the nested form with c_{j,k} = [q_j^-1]_{q_k}
  Signed handling (Sec. 5):            x > Q/2  ->  x - Q
"""
from __future__ import annotations

from math import prod


def rns_decompose(X: int, primes) -> list[int]:
    """x_i = X mod q_i (Sec. 2, RNS decomposition; also Sec. 5 limb-to-RNS projection)."""
    return [X % q for q in primes]


def crt_compose(residues, primes) -> int:
    """Eq. crt_composition, written out: the canonical X in [0, Q)."""
    Q = prod(primes)
    total = 0
    for x, q in zip(residues, primes):
        qhat = Q // q
        total += x * qhat * pow(qhat, -1, q)
    return total % Q


def garner_digits(residues, primes) -> list[int]:
    """Mixed-radix digits v_k of Eq. garner_mrc, evaluated in the nested order given there:

    v_k = | ((( x_k - v_0) c_{0,k} - v_1) c_{1,k} - ... - v_{k-1}) c_{k-1,k} |_{q_k}
    """
    v = []
    for k, (xk, qk) in enumerate(zip(residues, primes)):
        t = xk
        for j in range(k):
            t = (t - v[j]) * pow(primes[j], -1, qk) % qk
        v.append(t % qk)
    return v


def garner_compose(residues, primes) -> int:
    """X = sum_k v_k prod_{i<k} q_i from the digits (Eq. garner_mrc)."""
    v = garner_digits(residues, primes)
    X, w = 0, 1
    for vk, qk in zip(v, primes):
        X += vk * w
        w *= qk
    return X


def centered(x: int, Q: int) -> int:
    """Sec. 5 signed representation: for x in [0, Q), x > Q/2 becomes x - Q (Q/2 stays)."""
    x %= Q
    return x - Q if 2 * x > Q else x
