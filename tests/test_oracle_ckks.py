"""Pins for the oracle's CKKS scheme: decryption invariants (CPU only).

These fix the scheme's formulas independently of any implementation detail:
a dropped error term, a wrong sign in a key, a transposed operand in the
tensor product or a wrong rounding direction each breaks one of them.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, ckks, encode, ring

N_C1 = 1 << 11


def _setup(logN, logQ, logP, seed, hwt=None):
    g = fs.rng(seed)
    N = 1 << logN
    prm = ckks.CkksParams(logN, logQ, logP)
    s = [int(x) for x in (fs.sparse_ternary(g, N, hwt) if hwt else fs.ternary(g, (), N))]
    a_pk = bigint.from_limbs(fs.uniform_limbs(g, (), N, logQ))
    e_pk = [int(x) for x in fs.gaussian(g, (), N)]
    a_ev = bigint.from_limbs(fs.uniform_limbs(g, (), N, logQ + logP))
    e_ev = [int(x) for x in fs.gaussian(g, (), N)]
    pk = ckks.public_key(prm, s, a_pk, e_pk)
    evk = ckks.relin_key(prm, s, a_ev, e_ev)
    return g, prm, s, pk, evk


def _enc(g, prm, pk, m):
    N = prm.N
    v = [int(x) for x in fs.ternary(g, (), N)]
    e0 = [int(x) for x in fs.gaussian(g, (), N)]
    e1 = [int(x) for x in fs.gaussian(g, (), N)]
    return ckks.encrypt(prm, pk, m, v, e0, e1)


def test_public_key_relation():
    _, prm, s, pk, _ = _setup(8, 120, 120, 1)
    # b + a s = e (small) mod Q
    e = ckks.decrypt(s, pk, prm.logQ)
    assert max(abs(x) for x in e) <= fs.TAIL


def test_relin_key_relation():
    _, prm, s, _, evk = _setup(8, 120, 120, 2)
    # b' + a' s = e' + P s^2 (mod PQ)
    PQ = prm.P * prm.Q
    lhs = ring.mod_poly(ring.add_poly(evk[0], ring.negacyclic_mul(evk[1], s)), PQ)
    s2 = ring.negacyclic_mul(s, s)
    diff = [((x - prm.P * y) % PQ) for x, y in zip(lhs, s2)]
    diff = [d - PQ if 2 * d > PQ else d for d in diff]
    assert max(abs(d) for d in diff) <= fs.TAIL


def test_encrypt_decrypt_small_noise():
    g, prm, s, pk, _ = _setup(8, 120, 120, 3)
    m = [int(x) for x in fs.small_signed(g, (), prm.N, 40)]
    ct = _enc(g, prm, pk, m)
    dec = ckks.decrypt(s, ct, prm.logQ)
    # noise = v e + e0 + e1 s: |.| <= N*19 + 19 + N*19
    bound = 2 * prm.N * fs.TAIL + fs.TAIL
    assert max(abs(x - y) for x, y in zip(dec, m)) <= bound


def test_tensor_decrypts_to_product():
    g, prm, s, pk, _ = _setup(7, 100, 100, 4)
    m1 = [int(x) for x in fs.small_signed(g, (), prm.N, 20)]
    m2 = [int(x) for x in fs.small_signed(g, (), prm.N, 20)]
    c1 = _enc(g, prm, pk, m1)
    c2 = _enc(g, prm, pk, m2)
    d0, d1, d2 = ckks.tensor(c1, c2, prm.logQ)
    Q = prm.Q
    s2 = ring.negacyclic_mul(s, s)
    dec = ring.mod_poly(ring.add_poly(ring.add_poly(d0, ring.negacyclic_mul(d1, s)), ring.negacyclic_mul(d2, s2)), Q)
    dec = [x - Q if 2 * x > Q else x for x in dec]
    want = ring.negacyclic_mul(m1, m2)
    # error: e1 m2 + e2 m1 + e1 e2 with |e| <= 2 N 19 + 19
    eb = 2 * prm.N * fs.TAIL + fs.TAIL
    bound = 2 * prm.N * eb * (1 << 20) + prm.N * eb * eb
    assert max(abs(x - y) for x, y in zip(dec, want)) <= bound
    assert max(abs(x - y) for x, y in zip(dec, want)) < (1 << 40)  # far below |m1 m2| ~ 2^47


def test_relin_matches_three_component_decryption():
    g, prm, s, pk, evk = _setup(8, 120, 120, 5)
    m1 = [int(x) for x in fs.small_signed(g, (), prm.N, 30)]
    m2 = [int(x) for x in fs.small_signed(g, (), prm.N, 30)]
    c1 = _enc(g, prm, pk, m1)
    c2 = _enc(g, prm, pk, m2)
    d0, d1, d2 = ckks.tensor(c1, c2, prm.logQ)
    ct = ckks.relinearize(d0, d1, d2, evk, prm.logQ, prm.logP)
    Q = prm.Q
    s2 = ring.negacyclic_mul(s, s)
    three = ring.mod_poly(ring.add_poly(ring.add_poly(d0, ring.negacyclic_mul(d1, s)), ring.negacyclic_mul(d2, s2)), Q)
    two = ring.mod_poly(ring.add_poly(ct[0], ring.negacyclic_mul(ct[1], s)), Q)
    diff = [(x - y) % Q for x, y in zip(two, three)]
    diff = [d - Q if 2 * d > Q else d for d in diff]
    # key-switch error: (d2 e')/P + rounding: N Q 19 / P + (1 + N)/2 with P = Q
    bound = prm.N * fs.TAIL + (1 + prm.N)
    assert max(abs(d) for d in diff) <= bound


def test_rescale_rounds_half_up_and_divides():
    logQ = 64
    ct = ([0, 1, 2, 3, (1 << 64) - 1, 5 << 10], [1 << 9, (1 << 9) - 1, 3 << 9, 0, 7, 1 << 63])
    out = ckks.rescale(ct, 10, logQ)
    # round(x / 1024): 0, 0, 0, 0, round((2^64-1)/2^10) = 2^54 = 0 mod 2^54, 5
    assert out[0] == [0, 0, 0, 0, 0, 5]
    # 512/1024 = 0.5 -> 1 ; 511/1024 -> 0 ; 1536/1024 = 1.5 -> 2 ; 0 ; 7/1024 -> 0 ; 2^53
    assert out[1] == [1, 0, 2, 0, 0, 1 << 53]


def test_ckks_mult_accuracy_c1():
    """Decode(Dec(RS(Mult(Enc a, Enc b)))) ~= a*b within 2^-10 at scale 2^30 (N=2^11, Q=P=2^120)."""
    g, prm, s, pk, evk = _setup(11, 120, 120, 6)
    n = prm.N // 2
    z1 = fs.unit_disk(g, n)
    z2 = fs.unit_disk(g, n)
    m1 = encode.encode(z1, prm.N, 30)
    m2 = encode.encode(z2, prm.N, 30)
    c1 = _enc(g, prm, pk, m1)
    c2 = _enc(g, prm, pk, m2)
    ct = ckks.mult(c1, c2, evk, prm.logQ, prm.logP)
    ct = ckks.rescale(ct, 30, prm.logQ)
    dec = ckks.decrypt(s, ct, prm.logQ - 30)
    z = encode.decode(dec, prm.N, 30, n)
    err = np.abs(z - z1 * z2).max()
    assert err <= 2.0 ** -10 * max(1.0, np.abs(z1 * z2).max())


def test_rotation_shifts_slots_and_identity_step():
    g, prm, s, pk, _ = _setup(9, 120, 120, 7)
    n = prm.N // 2
    z = fs.unit_disk(g, n)
    m = encode.encode(z, prm.N, 40)
    ct = _enc(g, prm, pk, m)
    for step in (1, 4, n):  # step n = N/2: 5^(N/2) = 1 mod 2N, the identity automorphism
        a = bigint.from_limbs(fs.uniform_limbs(g, (), prm.N, prm.logQ + prm.logP))
        e = [int(x) for x in fs.gaussian(g, (), prm.N)]
        rtk = ckks.rotation_key(prm, s, step, a, e)
        out = ckks.rotate(ct, step, rtk, prm.N, prm.logQ, prm.logP)
        dec = encode.decode(ckks.decrypt(s, out, prm.logQ), prm.N, 40, n)
        want = np.roll(z, -step)
        assert np.abs(dec - want).max() < 2.0 ** -20
    assert ckks.galois_element(prm.N, n) == 1


def test_add_sub_negate_const():
    g, prm, s, pk, _ = _setup(6, 80, 80, 8)
    m1 = [int(x) for x in fs.small_signed(g, (), prm.N, 30)]
    m2 = [int(x) for x in fs.small_signed(g, (), prm.N, 30)]
    c1 = _enc(g, prm, pk, m1)
    c2 = _enc(g, prm, pk, m2)
    bound = 4 * prm.N * fs.TAIL + 2 * fs.TAIL
    for ct, want in ((ckks.add(c1, c2, prm.logQ), ring.add_poly(m1, m2)),
                     (ckks.sub(c1, c2, prm.logQ), ring.sub_poly(m1, m2)),
                     (ckks.negate(c1, prm.logQ), [-x for x in m1])):
        dec = ckks.decrypt(s, ct, prm.logQ)
        assert max(abs(x - y) for x, y in zip(dec, want)) <= bound
    dec = ckks.decrypt(s, ckks.mult_const(c1, -3, prm.logQ), prm.logQ)
    assert max(abs(x + 3 * y) for x, y in zip(dec, m1)) <= 3 * bound
    dec = ckks.decrypt(s, ckks.add_const(c1, 12345, prm.logQ), prm.logQ)
    assert abs(dec[0] - m1[0] - 12345) <= bound


def test_encode_constant_closed_form():
    # a real constant c in every slot encodes to round(c * Delta) at X^0 and zeros elsewhere
    N = 64
    m = encode.encode(np.full(N // 2, 0.75 + 0j), N, 20)
    assert m[0] == 786432 and all(x == 0 for x in m[1:])
    # decode(encode(z)) ~= z, and X -> X^5 rotates the slots left by one
    g = fs.rng(1)
    z = fs.unit_disk(g, N // 2)
    m = encode.encode(z, N, 40)
    assert np.abs(encode.decode(m, N, 40, N // 2) - z).max() < 2.0 ** -30
    rot = ring.automorphism(m, 5)
    assert np.abs(encode.decode(rot, N, 40, N // 2) - np.roll(z, -1)).max() < 2.0 ** -30


def test_moddown_by_hand_and_keeps_the_message():
    # moddownBy reduces every coefficient mod 2^logQ' (no division, the scale is unchanged)
    ct = ([5, (1 << 70) + 3, (1 << 80) - 1], [1 << 64, 7, (1 << 63) + 9])
    assert ckks.moddown(ct, 64) == ([5, 3, (1 << 64) - 1], [0, 7, (1 << 63) + 9])
    assert ckks.moddown(ct, 80) == (list(ct[0]), list(ct[1]))
    # Dec_{Q'}(ct mod Q') = Dec_Q(ct) while the message and noise stay below Q'/2
    g, prm, s, pk, _ = _setup(8, 120, 120, 9)
    m = [int(x) for x in fs.small_signed(g, (), prm.N, 30)]
    ct = _enc(g, prm, pk, m)
    bound = 2 * prm.N * fs.TAIL + fs.TAIL
    for lq in (97, 64, 33):
        dec = ckks.decrypt(s, ckks.moddown(ct, lq), lq)
        assert dec == ckks.decrypt(s, ct, prm.logQ)
        assert max(abs(x - y) for x, y in zip(dec, m)) <= bound


def _rotation_setup(seed, steps, logN=9, logQ=120, logP=120):
    g, prm, s, pk, evk = _setup(logN, logQ, logP, seed)
    rtk = {}
    for step in steps:
        a = bigint.from_limbs(fs.uniform_limbs(g, (), prm.N, prm.logQ + prm.logP))
        e = [int(x) for x in fs.gaussian(g, (), prm.N)]
        rtk[step] = ckks.rotation_key(prm, s, step, a, e)
    return g, prm, s, pk, evk, rtk


def test_negative_step_rotates_right():
    g, prm, s, pk, _, rtk = _rotation_setup(21, (-1, -5, 5, 1))
    n = prm.N // 2
    # 5 * 5^-1 = 1 mod 2N, and 5^-j 5^j = 1
    assert ckks.galois_element(prm.N, -1) * 5 % (2 * prm.N) == 1
    assert ckks.galois_element(prm.N, -5) * ckks.galois_element(prm.N, 5) % (2 * prm.N) == 1
    z = fs.unit_disk(g, n)
    ct = _enc(g, prm, pk, encode.encode(z, prm.N, 40))
    for step in (-1, -5):
        out = ckks.rotate(ct, step, rtk[step], prm.N, prm.logQ, prm.logP)
        dec = encode.decode(ckks.decrypt(s, out, prm.logQ), prm.N, 40, n)
        assert np.abs(dec - np.roll(z, -step)).max() < 2.0 ** -20  # right rotation: np.roll(z, +|step|)
    # rotating by -5 and then by +5 gives the slots back
    back = ckks.rotate(ckks.rotate(ct, -5, rtk[-5], prm.N, prm.logQ, prm.logP), 5, rtk[5], prm.N, prm.logQ, prm.logP)
    dec = encode.decode(ckks.decrypt(s, back, prm.logQ), prm.N, 40, n)
    assert np.abs(dec - z).max() < 2.0 ** -20


@pytest.mark.parametrize("logQl", [97, 64, 33])
def test_key_switching_below_the_top_level(logQl):
    """Relinearisation at a lower level Q_l with the top-level key (reduced mod P Q_l): the two-component
    decryption equals the three-component one up to the key-switch error, also at ragged levels."""
    g, prm, s, pk, evk = _setup(8, 120, 120, 30 + logQl)
    m1 = [int(x) for x in fs.small_signed(g, (), prm.N, 12)]
    m2 = [int(x) for x in fs.small_signed(g, (), prm.N, 12)]
    c1 = ckks.moddown(_enc(g, prm, pk, m1), logQl)
    c2 = ckks.moddown(_enc(g, prm, pk, m2), logQl)
    d0, d1, d2 = ckks.tensor(c1, c2, logQl)
    ct = ckks.relinearize(d0, d1, d2, evk, logQl, prm.logP)
    Q = 1 << logQl
    s2 = ring.negacyclic_mul(s, s)
    three = ring.mod_poly(ring.add_poly(ring.add_poly(d0, ring.negacyclic_mul(d1, s)), ring.negacyclic_mul(d2, s2)), Q)
    two = ring.mod_poly(ring.add_poly(ct[0], ring.negacyclic_mul(ct[1], s)), Q)
    diff = [(x - y) % Q for x, y in zip(two, three)]
    diff = [d - Q if 2 * d > Q else d for d in diff]
    # |d2 e'| / P + rounding <= N Q_l 19 / P + (1 + N) / 2 (P = 2^120 > Q_l)
    bound = prm.N * fs.TAIL * Q // prm.P + 1 + prm.N
    assert max(abs(d) for d in diff) <= bound
    # and a key for the wrong secret would not pass: the error would be of size Q_l
    if logQl >= 64:
        dec = ckks.decrypt(s, ct, logQl)
        want = ring.negacyclic_mul(m1, m2)
        assert max(abs(x - y) for x, y in zip(dec, want)) < 1 << 40


def test_rotation_below_the_top_level():
    g, prm, s, pk, _, rtk = _rotation_setup(22, (3,))
    n = prm.N // 2
    z = fs.unit_disk(g, n)
    ct = ckks.moddown(_enc(g, prm, pk, encode.encode(z, prm.N, 40)), 97)
    out = ckks.rotate(ct, 3, rtk[3], prm.N, 97, prm.logP)
    dec = encode.decode(ckks.decrypt(s, out, 97), prm.N, 40, n)
    assert np.abs(dec - np.roll(z, -3)).max() < 2.0 ** -20


def test_centred_representative_by_hand():
    Q = 1 << 8
    assert ckks.centred([0, 1, 127, 128, 129, 255, 256 + 3, -1], 8) == [0, 1, 127, -128, -127, -1, 3, -1]
    assert all(-Q // 2 <= x < Q // 2 for x in ckks.centred(list(range(-300, 300)), 8))


def test_rotation_adds_almost_no_error_at_scale_2_40():
    """Key switching the centred representative: a rotation's slots are as accurate as the fresh
    encryption's (N = 2^12, scale 2^40).  Key switching the [0, Q) representative instead makes the
    key error's mean term Q/2 (1 + X + ... + X^(N-1)) e' / P, whose slots grow like N, and fails this."""
    g, prm, s, pk, _, rtk = _rotation_setup(23, (1,), logN=12)
    n = prm.N // 2
    z = fs.unit_disk(g, n)
    ct = _enc(g, prm, pk, encode.encode(z, prm.N, 40))
    fresh = np.abs(encode.decode(ckks.decrypt(s, ct, prm.logQ), prm.N, 40, n) - z).max()
    out = ckks.rotate(ct, 1, rtk[1], prm.N, prm.logQ, prm.logP)
    rot = np.abs(encode.decode(ckks.decrypt(s, out, prm.logQ), prm.N, 40, n) - np.roll(z, -1)).max()
    assert rot <= 1.5 * fresh and rot < 2.0 ** -22


def test_conjugation_conjugates_every_slot():
    g, prm, s, pk, _ = _setup(9, 120, 120, 24)
    n = prm.N // 2
    a = bigint.from_limbs(fs.uniform_limbs(g, (), prm.N, prm.logQ + prm.logP))
    e = [int(x) for x in fs.gaussian(g, (), prm.N)]
    ck = ckks.conjugation_key(prm, s, a, e)
    # the key relation b' + a' s = e' + P s(X^-1) (mod P Q)
    PQ = prm.P * prm.Q
    lhs = ring.mod_poly(ring.add_poly(ck[0], ring.negacyclic_mul(ck[1], s)), PQ)
    sc = ring.automorphism(s, 2 * prm.N - 1)
    diff = ckks.centred([x - prm.P * y for x, y in zip(lhs, sc)], prm.logP + prm.logQ)
    assert max(abs(d) for d in diff) <= fs.TAIL
    z = fs.unit_disk(g, n)
    ct = _enc(g, prm, pk, encode.encode(z, prm.N, 40))
    out = ckks.conjugate(ct, ck, prm.N, prm.logQ, prm.logP)
    dec = encode.decode(ckks.decrypt(s, out, prm.logQ), prm.N, 40, n)
    assert np.abs(dec - np.conj(z)).max() < 2.0 ** -20
    # X -> X^(2N-1) on the plaintext alone conjugates the slots (closed form of the canonical embedding)
    m = encode.encode(z, prm.N, 40)
    assert np.abs(encode.decode(ring.automorphism(m, 2 * prm.N - 1), prm.N, 40, n) - np.conj(z)).max() < 2.0 ** -30


def test_imult_multiplies_slots_by_i():
    g, prm, s, pk, _ = _setup(9, 120, 120, 25)
    n = prm.N // 2
    z = fs.unit_disk(g, n)
    ct = _enc(g, prm, pk, encode.encode(z, prm.N, 40))
    out = ckks.imult(ct, prm.N, prm.logQ)
    dec = encode.decode(ckks.decrypt(s, out, prm.logQ), prm.N, 40, n)
    assert np.abs(dec - 1j * z).max() < 2.0 ** -20
    # i^2 = -1: imult twice is the negation, exactly (X^(N/2) X^(N/2) = X^N = -1)
    assert ckks.imult(out, prm.N, prm.logQ) == ckks.negate(ct, prm.logQ)


def test_mult_plain_multiplies_slots():
    g, prm, s, pk, _ = _setup(9, 160, 160, 26)
    n = prm.N // 2
    z1, z2 = fs.unit_disk(g, n), fs.unit_disk(g, n)
    ct = _enc(g, prm, pk, encode.encode(z1, prm.N, 40))
    m2 = encode.encode(z2, prm.N, 30)
    out = ckks.rescale(ckks.mult_plain(ct, m2, prm.logQ), 30, prm.logQ)
    dec = encode.decode(ckks.decrypt(s, out, prm.logQ - 30), prm.N, 40, n)
    assert np.abs(dec - z1 * z2).max() < 2.0 ** -20
    # closed forms: the constant 1 is the identity, X^(N/2) is imult, -1 is the negation
    one = [1] + [0] * (prm.N - 1)
    assert ckks.mult_plain(ct, one, prm.logQ) == tuple(list(p) for p in ct)
    half = [0] * prm.N
    half[prm.N // 2] = 1
    assert ckks.mult_plain(ct, half, prm.logQ) == ckks.imult(ct, prm.N, prm.logQ)
    assert ckks.mult_plain(ct, [-1] + [0] * (prm.N - 1), prm.logQ) == ckks.negate(ct, prm.logQ)
