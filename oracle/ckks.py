"""Non-RNS CKKS (HEAAN form) for the oracle (test infrastructure).

The paper names the operations (Sec. 6: keys sk, pk, rk, rtk; encrypt,
decrypt, mult with relinearisation, rescaleBy, moddownBy, leftrotate) and
adopts the original CKKS of Cheon et al. with HEAAN's parameterisation, but
prints no formulas.  This module writes out that scheme's standard
definitions, with Q = 2^logQ and the special modulus P = 2^logP:

  pk    = (b, a),   b = -a s + e            (mod Q)
  evk   = (b', a'), b' = -a' s + e' + P s^2  (mod P Q)
  rtk_j = (b', a'), b' = -a' s + e' + P s(X^(5^j))  (mod P Q)
  Enc(m; v, e0, e1) = (v b + m + e0, v a + e1)  (mod Q)
  Dec(b, a)         = [b + a s]_Q, centred (Sec. 5 signed handling)
  Mult: d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2 (mod Q), then
        (d0, d1) + round(P^-1 ([d2] b', [d2] a') mod P Q)  (mod Q)
  RS_k(c)  = round(c / 2^k)  (mod Q / 2^k)
  Rot_j(b, a) = (kappa(b), 0) + round(P^-1 kappa([a]) (b', a') mod P Q) (mod Q),
                kappa: X -> X^(5^j mod 2N) over Z
  Conj(b, a)  = the same with X -> X^(2N - 1) and the conjugation key

Readings where the paper is silent (recorded with the design notes):
  * round(y / 2^k) on the canonical representative y in [0, 2^K):
    floor((y + 2^(k-1)) / 2^k), i.e. halves round up;
  * ciphertexts at a lower level Q_l = 2^logQ_l use the top-level keys,
    reduced mod P Q_l (P Q_l divides P Q_top);
  * polynomials at rest are canonical representatives in [0, modulus);
  * the polynomial a key switch multiplies by the key is the centred
    representative [c] of c mod Q_l, in [-Q_l/2, Q_l/2) (c's logQ_l-bit two's
    complement; Sec. 5 signed handling), and a rotation applies kappa to [a]
    over Z, without reducing (kappa([a]) has coefficients in [-Q_l/2, Q_l/2]).
    The key-switch error is then |[c] e'| / P: with the [0, Q_l) representative
    its mean Q_l/2 multiplies e' by the all-ones polynomial, whose slots reach
    about 2N/pi, and a rotation at scale 2^40 misses the 2^-20 accuracy
    (measured 2^-17.6 at N = 2^15).  kappa over Z of [a] commutes with the
    transform, which allows hoisted rotations (Sec. 6 broadcast rotation).

Ring products go through ``ring.negacyclic_mul`` (exact over Z).
Parity: pinned by the decryption invariants in tests/test_oracle_ckks.py.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import ring


@dataclass(frozen=True)
class CkksParams:
    logN: int
    logQ: int
    logP: int

    @property
    def N(self) -> int:
        return 1 << self.logN

    @property
    def Q(self) -> int:
        return 1 << self.logQ

    @property
    def P(self) -> int:
        return 1 << self.logP


def _mul_mod(a, b, mod: int) -> list[int]:
    return ring.mod_poly(ring.negacyclic_mul(a, b), mod)


def round_shift(x: int, k: int) -> int:
    """round(x / 2^k) for x >= 0 with halves rounded up."""
    if k == 0:
        return x
    return (x + (1 << (k - 1))) >> k


def galois_element(N: int, step: int) -> int:
    """5^step mod 2N (left rotation by `step` slots); negative steps use 5^-1."""
    return pow(5, step, 2 * N)


def public_key(prm: CkksParams, s, a, e):
    Q = prm.Q
    b = ring.mod_poly(ring.add_poly(ring.scale_poly(ring.negacyclic_mul(a, s), -1), e), Q)
    return (b, ring.mod_poly(a, Q))


def switching_key(prm: CkksParams, s, s_from, a, e):
    """(b', a') with b' = -a' s + e' + P s_from (mod P Q): evk for s_from = s^2, rtk for kappa(s)."""
    PQ = prm.P * prm.Q
    t = ring.add_poly(ring.scale_poly(ring.negacyclic_mul(a, s), -1), e)
    t = ring.add_poly(t, ring.scale_poly(s_from, prm.P))
    return (ring.mod_poly(t, PQ), ring.mod_poly(a, PQ))


def relin_key(prm: CkksParams, s, a, e):
    return switching_key(prm, s, ring.negacyclic_mul(s, s), a, e)


def rotation_key(prm: CkksParams, s, step: int, a, e):
    g = galois_element(prm.N, step)
    return switching_key(prm, s, ring.automorphism(s, g), a, e)


def encrypt(prm: CkksParams, pk, m, v, e0, e1, logQ: int | None = None):
    """Enc at level logQ (default top): the pk is reduced mod 2^logQ."""
    Q = 1 << (prm.logQ if logQ is None else logQ)
    b = ring.mod_poly(ring.add_poly(ring.add_poly(ring.negacyclic_mul(v, pk[0]), m), e0), Q)
    a = ring.mod_poly(ring.add_poly(ring.negacyclic_mul(v, pk[1]), e1), Q)
    return (b, a)


def decrypt(s, ct, logQ: int):
    """Dec = [b + a s]_Q centred (Sec. 5 signed handling: x > Q/2 -> x - Q)."""
    Q = 1 << logQ
    raw = ring.mod_poly(ring.add_poly(ct[0], ring.negacyclic_mul(ct[1], s)), Q)
    return [x - Q if 2 * x > Q else x for x in raw]


def tensor(ct1, ct2, logQ: int):
    """(d0, d1, d2) = (b1 b2, a1 b2 + a2 b1, a1 a2) mod Q."""
    Q = 1 << logQ
    b1, a1 = ct1
    b2, a2 = ct2
    d0 = _mul_mod(b1, b2, Q)
    d1 = ring.mod_poly(ring.add_poly(ring.negacyclic_mul(a1, b2), ring.negacyclic_mul(a2, b1)), Q)
    d2 = _mul_mod(a1, a2, Q)
    return d0, d1, d2


def centred(c, logQ: int) -> list[int]:
    """The representative of c mod 2^logQ in [-2^(logQ-1), 2^(logQ-1))."""
    Q = 1 << logQ
    return [(int(x) % Q) - Q if (int(x) % Q) >= Q // 2 else int(x) % Q for x in c]


def key_switch(c, key, logQ: int, logP: int):
    """round(P^-1 (c b', c a') mod P Q_l) for an integer polynomial c (the caller picks its representative)."""
    PQ = 1 << (logP + logQ)
    Q = 1 << logQ
    yb = _mul_mod(c, key[0], PQ)
    ya = _mul_mod(c, key[1], PQ)
    return ([round_shift(x, logP) % Q for x in yb], [round_shift(x, logP) % Q for x in ya])


def relinearize(d0, d1, d2, evk, logQ: int, logP: int):
    Q = 1 << logQ
    kb, ka = key_switch(centred(d2, logQ), evk, logQ, logP)
    return (ring.mod_poly(ring.add_poly(d0, kb), Q), ring.mod_poly(ring.add_poly(d1, ka), Q))


def mult(ct1, ct2, evk, logQ: int, logP: int):
    """Homomorphic multiplication with relinearisation (mult_pairwise_into, Sec. 6)."""
    d0, d1, d2 = tensor(ct1, ct2, logQ)
    return relinearize(d0, d1, d2, evk, logQ, logP)


def rescale(ct, k: int, logQ: int):
    """rescaleBy (Sec. 6): round(c / 2^k) mod 2^(logQ - k)."""
    Qn = 1 << (logQ - k)
    return tuple([round_shift(x, k) % Qn for x in poly] for poly in ct)


def moddown(ct, new_logQ: int):
    """moddownBy (Sec. 6) for CKKS: reduce mod 2^new_logQ (the scale is unchanged)."""
    Qn = 1 << new_logQ
    return tuple([x % Qn for x in poly] for poly in ct)


def apply_automorphism(ct, g: int, key, logQ: int, logP: int):
    """(kappa_g(b), 0) + key switch of kappa_g([a]) (over Z) back to s, mod Q."""
    Q = 1 << logQ
    kb = ring.mod_poly(ring.automorphism(ct[0], g), Q)
    ka = ring.automorphism(centred(ct[1], logQ), g)
    sb, sa = key_switch(ka, key, logQ, logP)
    return (ring.mod_poly(ring.add_poly(kb, sb), Q), sa)


def rotate(ct, step: int, rtk, N: int, logQ: int, logP: int):
    """leftrotate (Sec. 6): kappa_{5^step} then key switch back to s."""
    return apply_automorphism(ct, galois_element(N, step), rtk, logQ, logP)


def conjugation_key(prm: CkksParams, s, a, e):
    """ck (Sec. 6 conjugation key): the switching key of s(X^(2N-1))."""
    return switching_key(prm, s, ring.automorphism(s, 2 * prm.N - 1), a, e)


def conjugate(ct, ck, N: int, logQ: int, logP: int):
    """conjugate_pairwise_into (Sec. 6): X -> X^(2N-1) conjugates every slot, then key switch."""
    return apply_automorphism(ct, 2 * N - 1, ck, logQ, logP)


def add(ct1, ct2, logQ: int):
    Q = 1 << logQ
    return tuple(ring.mod_poly(ring.add_poly(x, y), Q) for x, y in zip(ct1, ct2))


def sub(ct1, ct2, logQ: int):
    Q = 1 << logQ
    return tuple(ring.mod_poly(ring.sub_poly(x, y), Q) for x, y in zip(ct1, ct2))


def negate(ct, logQ: int):
    Q = 1 << logQ
    return tuple([(-x) % Q for x in poly] for poly in ct)


def mult_const(ct, c: int, logQ: int):
    """Ciphertext times an integer constant (multconst with an integer-encoded scalar)."""
    Q = 1 << logQ
    return tuple([(x * c) % Q for x in poly] for poly in ct)


def imult(ct, N: int, logQ: int):
    """imult (Sec. 6): both polynomials times X^(N/2), the imaginary unit at every slot (5^j = 1 mod 4)."""
    Q = 1 << logQ
    mono = [0] * N
    mono[N // 2] = 1
    return tuple(ring.mod_poly(ring.negacyclic_mul(poly, mono), Q) for poly in ct)


def mult_plain(ct, m, logQ: int):
    """multconstvec (Sec. 6): both polynomials times the plaintext polynomial m, mod Q."""
    Q = 1 << logQ
    return tuple(_mul_mod(poly, m, Q) for poly in ct)


def add_const(ct, c: int, logQ: int):
    """Add an integer constant to the constant coefficient of b (addconst)."""
    Q = 1 << logQ
    b = list(ct[0])
    b[0] = (b[0] + c) % Q
    return (b, list(ct[1]))
