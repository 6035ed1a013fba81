"""Non-RNS BGV with an odd modulus chain, for the oracle (test infrastructure).

The paper runs one CKKS-BGV abstraction (Sec. 6 "unified CKKS-BGV scheme
abstraction") but prints no BGV formulas or modulus chain.  This module
writes out the standard BGV definitions on a single big odd modulus:

  chain       Q_l = q0 r^l (l = 0..L), q0 and r odd, q0 = r = 1 (mod t)
  special     P = 2^logP, coprime to t
  pk          (b, a),   b = -a s + t e                  (mod Q_L)
  evk         (b', a'), b' = -a' s + t e' + P s^2         (mod P Q_L)
  Enc(m)      (v b + m + t e0, v a + t e1)             (mod Q_l)
  Dec         [[b + a s]_{Q_l}]_t  (centred mod Q_l, then mod t)
  Mult        (d0, d1, d2) = (b1 b2, a1 b2 + a2 b1, a1 a2) mod Q_l, then
              (d0, d1) + KS(d2 b', d2 a') mod Q_l
  KS(y)       (y + delta) / P with delta = t [(-y) t^-1]_P  (centred mod P):
              y + delta = 0 (mod P), delta = 0 (mod t), |delta| <= t P / 2
  ModSwitch   Q_l -> Q_{l-1} = Q_l / r: c' = (c + delta') / r, delta' =
              t [(-c) t^-1]_r (centred mod r); r = 1 (mod t) keeps m

Readings (recorded with the design notes): centred residues use the
half-open range [-m/2, m/2) for even m and (-m/2, m/2) for odd m; all
polynomials at rest are canonical residues in [0, modulus); the key switch
uses the top-level key reduced implicitly (P Q_l divides P Q_L).
Parity: pinned by the exact plaintext invariant m^(2^k) mod (X^N + 1, t)
after every step of a squaring chain (tests/test_oracle_bgv.py).
"""
from __future__ import annotations

from dataclasses import dataclass

from . import ring


def centred(x: int, m: int) -> int:
    """Representative of x mod m in [-m/2, m/2) (m even) or (-m/2, m/2) (m odd)."""
    x %= m
    return x - m if 2 * x >= m else x


@dataclass(frozen=True)
class BgvParams:
    logN: int
    t: int
    q0: int
    r: int
    levels: int
    logP: int

    @property
    def N(self) -> int:
        return 1 << self.logN

    @property
    def P(self) -> int:
        return 1 << self.logP

    def Q(self, level: int) -> int:
        return self.q0 * self.r ** level

    @property
    def Qtop(self) -> int:
        return self.Q(self.levels)


def chain_moduli(t: int, log_q0: int, log_r: int) -> tuple[int, int]:
    """q0 ~ 2^log_q0 and r ~ 2^log_r, odd and = 1 (mod t): the largest such values below the powers of two."""
    def pick(bits):
        k = ((1 << bits) - 1) // t
        if (1 + t * k) % 2 == 0:
            k -= 1
        return 1 + t * k

    return pick(log_q0), pick(log_r)


def public_key(prm: BgvParams, s, a, e):
    Q = prm.Qtop
    b = ring.mod_poly(ring.add_poly(ring.scale_poly(ring.negacyclic_mul(a, s), -1), ring.scale_poly(e, prm.t)), Q)
    return (b, ring.mod_poly(a, Q))


def relin_key(prm: BgvParams, s, a, e):
    PQ = prm.P * prm.Qtop
    t = ring.add_poly(ring.scale_poly(ring.negacyclic_mul(a, s), -1), ring.scale_poly(e, prm.t))
    t = ring.add_poly(t, ring.scale_poly(ring.negacyclic_mul(s, s), prm.P))
    return (ring.mod_poly(t, PQ), ring.mod_poly(a, PQ))


def encrypt(prm: BgvParams, pk, m, v, e0, e1, level: int | None = None):
    Q = prm.Q(prm.levels if level is None else level)
    t = prm.t
    b = ring.add_poly(ring.add_poly(ring.negacyclic_mul(v, pk[0]), m), ring.scale_poly(e0, t))
    a = ring.add_poly(ring.negacyclic_mul(v, pk[1]), ring.scale_poly(e1, t))
    return (ring.mod_poly(b, Q), ring.mod_poly(a, Q))


def decrypt(prm: BgvParams, s, ct, level: int) -> list[int]:
    """[[b + a s]_{Q_l}]_t with the centred representative mod Q_l, result in [0, t)."""
    Q = prm.Q(level)
    raw = ring.add_poly(ct[0], ring.negacyclic_mul(ct[1], s))
    return [centred(x, Q) % prm.t for x in raw]


def key_switch_divide(y: int, prm: BgvParams) -> int:
    """(y + delta) / P with delta = t [(-y) t^-1]_P: exact division, a multiple of t added."""
    P, t = prm.P, prm.t
    u = centred(-y * pow(t, -1, P), P)
    delta = t * u
    assert (y + delta) % P == 0
    return (y + delta) // P


def mult(prm: BgvParams, ct1, ct2, evk, level: int):
    """Homomorphic multiplication with relinearisation at level `level`."""
    Q = prm.Q(level)
    PQ = prm.P * Q
    b1, a1 = ct1
    b2, a2 = ct2
    d0 = ring.mod_poly(ring.negacyclic_mul(b1, b2), Q)
    d1 = ring.mod_poly(ring.add_poly(ring.negacyclic_mul(a1, b2), ring.negacyclic_mul(a2, b1)), Q)
    d2 = ring.mod_poly(ring.negacyclic_mul(a1, a2), Q)
    yb = ring.mod_poly(ring.negacyclic_mul(d2, evk[0]), PQ)
    ya = ring.mod_poly(ring.negacyclic_mul(d2, evk[1]), PQ)
    cb = [(x + key_switch_divide(y, prm)) % Q for x, y in zip(d0, yb)]
    ca = [(x + key_switch_divide(y, prm)) % Q for x, y in zip(d1, ya)]
    return (cb, ca)


def mod_switch(prm: BgvParams, ct, level: int):
    """Q_level -> Q_{level-1} = Q_level / r (moddownBy for BGV)."""
    r, t = prm.r, prm.t
    Qn = prm.Q(level - 1)
    out = []
    for poly in ct:
        res = []
        for c in poly:
            d = t * centred(-c * pow(t, -1, r), r)
            assert (c + d) % r == 0
            res.append(((c + d) // r) % Qn)
        out.append(res)
    return tuple(out)


def plaintext_power(m, k: int, N: int, t: int) -> list[int]:
    """m^(2^k) in Z_t[X]/(X^N + 1) by k plain squarings."""
    x = [int(v) % t for v in m]
    for _ in range(k):
        x = ring.mod_poly(ring.negacyclic_mul(x, x), t)
    return x


def primitive_root(t: int) -> int:
    """The smallest generator of the multiplicative group mod the prime t."""
    r, fac, d = t - 1, [], 2
    while d * d <= r:
        if r % d == 0:
            fac.append(d)
            while r % d == 0:
                r //= d
        d += 1
    if r > 1:
        fac.append(r)
    g = 2
    while any(pow(g, (t - 1) // p, t) == 1 for p in fac):
        g += 1
    return g


def slot_root(N: int, t: int) -> int:
    """psi = g^((t-1)/(2N)): a primitive 2N-th root of unity mod t (needs t = 1 mod 2N)."""
    assert (t - 1) % (2 * N) == 0
    return pow(primitive_root(t), (t - 1) // (2 * N), t)


def slot_decode(m, N: int, t: int) -> list[int]:
    """Slots of a plaintext (Sec. 2 polynomial CRT): slot k = m(psi^(2k+1)) mod t, by the direct sum."""
    psi = slot_root(N, t)
    out = []
    for k in range(N):
        x = pow(psi, 2 * k + 1, t)
        acc, p = 0, 1
        for j in range(N):
            acc = (acc + int(m[j]) * p) % t
            p = p * x % t
        out.append(acc)
    return out


def slot_encode(slots, N: int, t: int) -> list[int]:
    """The plaintext whose slots are `slots`: m_j = N^-1 sum_k slots_k psi^(-(2k+1) j) mod t (inverse of the
    evaluation at the N distinct roots psi^(2k+1) of X^N + 1)."""
    psi_inv = pow(slot_root(N, t), t - 2, t)
    n_inv = pow(N, t - 2, t)
    out = []
    for j in range(N):
        acc = 0
        for k in range(N):
            acc = (acc + int(slots[k]) * pow(psi_inv, (2 * k + 1) * j, t)) % t
        out.append(acc * n_inv % t)
    return out

