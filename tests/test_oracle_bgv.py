"""Pins for the oracle's BGV scheme (CPU only).

The exact invariant: after every multiplication, relinearisation and modulus
switch of a squaring chain, decryption equals m^(2^k) in Z_t[X]/(X^N + 1),
computed with plain arithmetic mod t.  Any wrong sign in a key, a dropped
error term, a mis-centred delta or a wrong modulus breaks it.
"""
import pytest

import fhe_synth as fs
from oracle import bgv, bigint, ring

T = 65537


def test_chain_moduli_form():
    q0, r = bgv.chain_moduli(T, 54, 48)
    assert q0 % 2 == 1 and r % 2 == 1
    assert q0 % T == 1 and r % T == 1
    assert q0 < (1 << 54) and q0 > (1 << 54) - 2 * T
    assert r < (1 << 48) and r > (1 << 48) - 2 * T
    prm = bgv.BgvParams(14, T, q0, r, 8, 438)
    assert prm.Qtop.bit_length() == 438  # logQ = 54 + 8 * 48


def test_centred_ranges():
    assert bgv.centred(7, 16) == 7 and bgv.centred(8, 16) == -8 and bgv.centred(9, 16) == -7
    assert bgv.centred(7, 15) == 7 and bgv.centred(8, 15) == -7
    assert bgv.centred(-1, 10) == -1


def test_key_switch_divide_by_hand():
    prm = bgv.BgvParams(3, 7, 1, 1, 0, 4)  # t = 7, P = 16
    # y = 5: t^-1 mod 16 = 7; -5 * 7 = -35 = 13 mod 16 -> centred -3; delta = -21; (5 - 21)/16 = -1
    assert bgv.key_switch_divide(5, prm) == -1
    for y in range(-200, 200):
        z = bgv.key_switch_divide(y, prm)
        d = z * 16 - y
        assert d % 7 == 0 and abs(d) <= 7 * 8


def _setup(logN, levels, seed):
    q0, r = bgv.chain_moduli(T, 54, 48)
    prm = bgv.BgvParams(logN, T, q0, r, levels, 54 + 48 * levels)
    g = fs.rng(seed)
    N = prm.N
    s = [int(x) for x in fs.ternary(g, (), N)]
    Qbits = prm.Qtop.bit_length()
    a = [x % prm.Qtop for x in bigint.from_limbs(fs.uniform_limbs(g, (), N, Qbits + 64))]
    pk = bgv.public_key(prm, s, a, [int(x) for x in fs.gaussian(g, (), N)])
    PQ = prm.P * prm.Qtop
    a2 = [x % PQ for x in bigint.from_limbs(fs.uniform_limbs(g, (), N, PQ.bit_length() + 64))]
    evk = bgv.relin_key(prm, s, a2, [int(x) for x in fs.gaussian(g, (), N)])
    return g, prm, s, pk, evk


def test_key_relations():
    g, prm, s, pk, evk = _setup(6, 3, 1)
    Q, PQ = prm.Qtop, prm.P * prm.Qtop
    e = [bgv.centred(x, Q) for x in ring.add_poly(pk[0], ring.negacyclic_mul(pk[1], s))]
    assert all(x % T == 0 and abs(x) <= T * fs.TAIL for x in e)
    lhs = ring.add_poly(evk[0], ring.negacyclic_mul(evk[1], s))
    s2 = ring.negacyclic_mul(s, s)
    e2 = [bgv.centred(x - prm.P * y, PQ) for x, y in zip(lhs, s2)]
    assert all(x % T == 0 and abs(x) <= T * fs.TAIL for x in e2)


@pytest.mark.parametrize("logN,levels", [(5, 3), (8, 8)])
def test_squaring_chain_decrypts_exactly(logN, levels):
    g, prm, s, pk, evk = _setup(logN, levels, 10 + logN)
    N = prm.N
    m = [int(x) for x in fs.uniform_mod_t(g, (), N, T)]
    ct = bgv.encrypt(prm, pk, m, [int(x) for x in fs.ternary(g, (), N)], [int(x) for x in fs.gaussian(g, (), N)],
                     [int(x) for x in fs.gaussian(g, (), N)])
    assert bgv.decrypt(prm, s, ct, levels) == m
    for k in range(1, levels + 1):
        level = levels - k + 1
        ct = bgv.mult(prm, ct, ct, evk, level)
        assert bgv.decrypt(prm, s, ct, level) == bgv.plaintext_power(m, k, N, T), f"mult {k}"
        ct = bgv.mod_switch(prm, ct, level)
        assert bgv.decrypt(prm, s, ct, level - 1) == bgv.plaintext_power(m, k, N, T), f"modswitch {k}"


def test_mod_switch_by_hand():
    # t = 3, r = 7 (= 1 mod 3), q0 = 4: Q_1 = 28, Q_0 = 4.
    # c = 5:  t^-1 mod 7 = 5; -5*5 = -25 = 3 (mod 7), centred 3; delta = 9; (5 + 9)/7 = 2
    # c = 20: -20*5 = -100 = 5 (mod 7), centred -2; delta = -6; (20 - 6)/7 = 2
    prm = bgv.BgvParams(1, 3, 4, 7, 1, 3)
    out = bgv.mod_switch(prm, ([5, 20], [0, 0]), 1)
    assert out[0] == [2, 2]


def test_slot_maps_by_hand_and_as_ring_isomorphism():
    """Sec. 2 polynomial CRT: N = 4, t = 17 (2N = 8 divides 16): g = 3, psi = 3^2 = 9 (9^4 = -1 mod 17);
    the slots of 1 + X are 1 + 9^(2k+1) = 10, 16, 9, 3.  Slot-wise products are ring products."""
    assert bgv.primitive_root(17) == 3 and bgv.slot_root(4, 17) == 9
    assert bgv.slot_decode([1, 1, 0, 0], 4, 17) == [10, 16, 9, 3]
    assert bgv.slot_encode([10, 16, 9, 3], 4, 17) == [1, 1, 0, 0]
    import fhe_synth as fs
    from oracle import ring

    t, N = 65537, 64
    g = fs.rng(71)
    x = [int(v) for v in fs.uniform_mod_t(g, (), N, t)]
    y = [int(v) for v in fs.uniform_mod_t(g, (), N, t)]
    mx, my = bgv.slot_encode(x, N, t), bgv.slot_encode(y, N, t)
    assert bgv.slot_decode(mx, N, t) == x
    prod = ring.mod_poly(ring.negacyclic_mul(mx, my), t)
    assert bgv.slot_decode(prod, N, t) == [a * b % t for a, b in zip(x, y)]
    assert bgv.primitive_root(65537) == 3
