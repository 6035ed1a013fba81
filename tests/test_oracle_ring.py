"""Pins for the oracle's ring arithmetic, NTT definitions and CRT (CPU only).

Each check ties the oracle to something other than itself: hand-worked
fixtures from the paper's equations, closed forms, textbook identities and
brute force on small inputs.
"""
import os

import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, crt, ntt, ring

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([[int(t) for t in part.split()] for part in line.split("|")])
    return rows


@pytest.mark.parametrize("mul", [ring.negacyclic_schoolbook, ring.negacyclic_kronecker, ring.negacyclic_fast])
def test_negacyclic_golden(mul):
    for (n,), a, b, c in _read_rows("negacyclic_small.txt"):
        assert len(a) == n and len(b) == n
        assert mul(a, b) == c


def _rand_poly(g, n, bits, signed=True):
    limbs = fs.uniform_limbs(g, (), n, bits)
    vals = bigint.from_limbs(limbs)
    if signed:
        sg = g.integers(0, 2, size=n)
        vals = [-v if s else v for v, s in zip(vals, sg)]
    return vals


def test_monomial_closed_form():
    # (c X^i)(d X^j) = c d X^(i+j) if i+j < N else -c d X^(i+j-N)
    N = 16
    for i in range(N):
        for j in range(N):
            a = [0] * N
            b = [0] * N
            a[i] = 7
            b[j] = -3
            want = [0] * N
            e = i + j
            if e < N:
                want[e] = -21
            else:
                want[e - N] = 21
            assert ring.negacyclic_schoolbook(a, b) == want


def test_identity_and_negation():
    g = fs.rng(11)
    N = 128
    a = _rand_poly(g, N, 200)
    one = [1] + [0] * (N - 1)
    minus_one = [-1] + [0] * (N - 1)
    for mul in (ring.negacyclic_kronecker, ring.negacyclic_fast):
        assert mul(a, one) == a
        assert mul(one, a) == a
        assert mul(a, minus_one) == [-x for x in a]


@pytest.mark.parametrize("N,bits", [(32, 64), (256, 120), (1024, 37)])
def test_three_products_agree(N, bits):
    g = fs.rng(100 + N)
    a = _rand_poly(g, N, bits)
    b = _rand_poly(g, N, bits + 13)
    ref = ring.negacyclic_schoolbook(a, b)
    assert ring.negacyclic_kronecker(a, b) == ref
    assert ring.negacyclic_fast(a, b) == ref


def test_fast_matches_schoolbook_c1_size():
    # N = 2^11 with 120-bit operands: the size of the smallest workload
    g = fs.rng(7)
    N = 2048
    a = bigint.from_limbs(fs.uniform_limbs(g, (), N, 120))
    b = bigint.from_limbs(fs.uniform_limbs(g, (), N, 120))
    assert ring.negacyclic_fast(a, b) == ring.negacyclic_schoolbook(a, b)


def test_fast_matches_kronecker_4096():
    g = fs.rng(8)
    N = 4096
    a = _rand_poly(g, N, 300)
    b = _rand_poly(g, N, 1000)
    assert ring.negacyclic_fast(a, b) == ring.negacyclic_kronecker(a, b)


def test_fast_truncated_output_is_mod_power_of_two():
    g = fs.rng(9)
    N = 256
    a = _rand_poly(g, N, 150)
    b = _rand_poly(g, N, 150)
    exact = ring.negacyclic_kronecker(a, b)
    got = ring.negacyclic_fast(a, b, out_bits=96)
    assert [x % (1 << 96) for x in got] == [x % (1 << 96) for x in exact]


def test_automorphism_is_ring_homomorphism():
    g = fs.rng(12)
    N = 64
    a = _rand_poly(g, N, 40)
    b = _rand_poly(g, N, 40)
    for gal in (5, 25, 2 * N - 1, 3):
        lhs = ring.automorphism(ring.negacyclic_schoolbook(a, b), gal)
        rhs = ring.negacyclic_schoolbook(ring.automorphism(a, gal), ring.automorphism(b, gal))
        assert lhs == rhs
    # X -> X^g on a monomial, by hand: X^3 with g = 5, N = 4: X^15 = X^(15-8) * X^8 = X^7 = -X^3
    assert ring.automorphism([0, 0, 0, 1], 5) == [0, 0, 0, -1]
    # g = 1 is the identity
    assert ring.automorphism(a, 1) == a


def test_limb_roundtrip_and_layout():
    vals = [0, 1, (1 << 32) + 5, (1 << 64) - 1, -1, -(1 << 40)]
    L = 3
    limbs = bigint.to_limbs(vals, L)
    assert limbs.shape == (L, len(vals))
    assert limbs[0, 2] == 5 and limbs[1, 2] == 1 and limbs[2, 2] == 0
    assert limbs[0, 4] == 0xFFFFFFFF and limbs[2, 4] == 0xFFFFFFFF
    assert bigint.from_limbs(limbs, signed=True) == vals
    assert bigint.from_limbs(limbs)[4] == (1 << 96) - 1


# ------------------------------------------------------------------ NTT


@pytest.mark.parametrize("N", [8, 32])
def test_ntt_closed_forms(N):
    q = ntt.ntt_primes(1, 2 * N)[0]
    psi = ntt.primitive_2n_root(q, N)
    assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1
    # NTT(X^k)_i = psi^((2i+1)k)  (Eq. negacyclic_ntt with a single term)
    for k in range(N):
        mono = [0] * N
        mono[k] = 1
        assert ntt.ntt_direct(mono, q, psi) == [pow(psi, (2 * i + 1) * k, q) for i in range(N)]
    # the constant 1 maps to all ones
    assert ntt.ntt_direct([1] + [0] * (N - 1), q, psi) == [1] * N
    # iNTT o NTT = id (Eq. negacyclic_intt inverts Eq. negacyclic_ntt)
    g = fs.rng(N)
    a = [int(x) for x in g.integers(0, q, size=N)]
    assert ntt.intt_direct(ntt.ntt_direct(a, q, psi), q, psi) == a


def test_ntt_product_matches_schoolbook():
    N = 32
    q = ntt.ntt_primes(2, 2 * N)[1]
    psi = ntt.primitive_2n_root(q, N)
    g = fs.rng(3)
    a = [int(x) for x in g.integers(0, q, size=N)]
    b = [int(x) for x in g.integers(0, q, size=N)]
    want = ring.mod_poly(ring.negacyclic_schoolbook(a, b), q)
    assert ntt.ntt_mul_mod_q(a, b, q, psi) == want


def test_ntt_primes_form():
    ps = ntt.ntt_primes(20, 1 << 17)
    assert all((p - 1) % (1 << 17) == 0 and (1 << 30) < p < (1 << 31) for p in ps)
    assert ps == sorted(ps, reverse=True) and len(set(ps)) == 20
    assert all(ntt.is_prime(p) for p in ps)
    assert not ntt.is_prime(561) and not ntt.is_prime(2147483649)  # Carmichael, 3*715827883


# ------------------------------------------------------------------ CRT


def test_garner_golden():
    for primes, res, digits, (X,) in _read_rows("garner_small.txt"):
        assert crt.rns_decompose(X, primes) == res
        assert crt.garner_digits(res, primes) == digits
        assert crt.garner_compose(res, primes) == X
        assert crt.crt_compose(res, primes) == X


def test_crt_and_garner_random():
    primes = ntt.ntt_primes(12, 1 << 12)
    M = 1
    for p in primes:
        M *= p
    g = fs.rng(5)
    for _ in range(200):
        X = int(bigint.from_limbs(fs.uniform_limbs(g, (), 1, 400))[0]) % M
        r = crt.rns_decompose(X, primes)
        assert crt.crt_compose(r, primes) == X
        assert crt.garner_compose(r, primes) == X
        # negatives: the residues of M - X compose to M - X, centred to -X
        rn = crt.rns_decompose(-X, primes)
        assert crt.centered(crt.garner_compose(rn, primes), M) == (-X if 2 * X < M else M - X)


def test_centered_tie_and_range():
    assert crt.centered(8, 16) == 8  # x = Q/2 stays positive (strict '>')
    assert crt.centered(9, 16) == -7
    assert crt.centered(7, 15) == 7 and crt.centered(8, 15) == -7


# ---- the exact product at the operand widths of the key switch at N = 2^16, logQ = logP = 1200 (and 1550):
# d2 (logQ bits) times a key polynomial (logP + logQ bits) needs about 3,616 bits and ~60 62-bit primes in
# fastmul.c; these regimes are checked against schoolbook, Kronecker and a closed form.

@pytest.mark.parametrize("bits_a,bits_b", [(1200, 1200), (2400, 2400), (1200, 2400), (1550, 3100)])
def test_fast_matches_schoolbook_at_key_switch_widths(bits_a, bits_b):
    g = fs.rng(bits_a + bits_b)
    N = 64
    a = _rand_poly(g, N, bits_a)
    b = _rand_poly(g, N, bits_b)
    assert ring.negacyclic_fast(a, b) == ring.negacyclic_schoolbook(a, b)


def test_fast_matches_kronecker_4096_at_key_switch_widths():
    """N = 2^12 with 1,200 x 2,400-bit operands: a 3,600-bit product bound (takes ~15 s in Kronecker form)."""
    g = fs.rng(10)
    N = 4096
    a = _rand_poly(g, N, 1200)
    b = _rand_poly(g, N, 2400)
    assert ring.negacyclic_fast(a, b) == ring.negacyclic_kronecker(a, b)


def test_fast_binomial_closed_form_at_full_ring():
    """N = 2^16: a full 1,200-bit polynomial times c X^i + d X^j (2,400-bit c, d) is the sum of two
    negacyclic shifts, c X^i a + d X^j a; a wrong NTT length, root or CRT width fails it."""
    g = fs.rng(11)
    N = 1 << 16
    a = _rand_poly(g, N, 1200)
    c, d = _rand_poly(g, 2, 2400)
    i, j = 1, N - 3
    b = [0] * N
    b[i], b[j] = c, d

    def shift(v, k, m):  # m X^k v(X) in Z[X]/(X^N + 1)
        return [m * (v[n - k] if n >= k else -v[n - k + N]) for n in range(N)]

    want = [x + y for x, y in zip(shift(a, i, c), shift(a, j, d))]
    assert ring.negacyclic_fast(a, b) == want
