"""GPU path vs the CPU oracle, bit for bit, through the C ABI (needs a GB300).

Sizes: small rings where the oracle is quick but which still span several
tiles, levels with a ragged top limb (logQ not a multiple of 32) and exact
multiples, uniform full-range ciphertexts, zeros and all-ones, batches
(cnum > 1), and one full-size case at N = 2^16, logQ = logP = 1200 in the
bench's launch configuration.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, ckks, encode, ring

from fhe_setup import ct_ints, encrypt_both, make_pair, random_ct_limbs, to_dev

pytestmark = pytest.mark.gpu


def _ct_from_limbs(P, limbs, logQ):
    import paper_2607_05920_gb300 as fhe

    return fhe.Ciphertext(to_dev(limbs), logQ)


def _oracle_ct(limbs):
    return [tuple(bigint.from_limbs(limbs[c, p]) for p in range(2)) for c in range(limbs.shape[0])]


@pytest.mark.parametrize("crt", [0, 1, 2, 3], ids=["direct_tc", "garner", "direct_int", "direct_tc_cvt"])
@pytest.mark.parametrize("logN,La,Lb,logOut", [(11, 4, 4, 268), (11, 3, 1, 100), (8, 1, 1, 64), (14, 5, 7, 200),
                                                (16, 2, 3, 64), (12, 40, 40, 2600)])
def test_ring_mul_matches_exact_product(logN, La, Lb, logOut, crt):
    import paper_2607_05920_gb300 as fhe

    ctx = fhe.Context(logN, 1300, 1300, crt=crt)
    g = fs.rng(logN * 100 + La)
    N = 1 << logN
    cnum = 2
    a = fs.uniform_limbs(g, (cnum,), N, 32 * La)
    b = fs.uniform_limbs(g, (cnum,), N, 32 * Lb)
    if logN == 8:  # extremes: all-ones operands and a zero operand
        a[0][:] = 0xFFFFFFFF
        b[0][:] = 0xFFFFFFFF
        b[1][:] = 0
    out = ctx.ring_mul(to_dev(a), to_dev(b), logOut).cpu().numpy().view(np.uint32)
    for c in range(cnum):
        want = ring.negacyclic_fast(bigint.from_limbs(a[c]), bigint.from_limbs(b[c]))
        got = bigint.from_limbs(out[c])
        assert got == [x % (1 << logOut) for x in want]
    ctx.close()


@pytest.mark.parametrize("crt", [0, 1, 2, 3], ids=["direct_tc", "garner", "direct_int", "direct_tc_cvt"])
def test_ring_mul_every_limb_bucket(crt):
    """Outputs of 8 .. 128 limbs (every register bucket of the reconstruction), products wider than the output."""
    import paper_2607_05920_gb300 as fhe

    logN = 8
    N = 1 << logN
    ctx = fhe.Context(logN, 2000, 1900, crt=crt)
    g = fs.rng(88 + crt)
    for out_limbs in (8, 13, 16, 24, 32, 38, 40, 48, 56, 64, 75, 80, 96, 112, 128):
        logOut = 32 * out_limbs - 5
        La = out_limbs // 2 + 1
        a = fs.uniform_limbs(g, (1,), N, 32 * La)
        b = fs.uniform_limbs(g, (1,), N, 32 * La - 7)
        out = ctx.ring_mul(to_dev(a), to_dev(b), logOut).cpu().numpy().view(np.uint32)
        want = ring.negacyclic_fast(bigint.from_limbs(a[0]), bigint.from_limbs(b[0]))
        assert bigint.from_limbs(out[0]) == [x % (1 << logOut) for x in want], out_limbs
    ctx.close()


@pytest.fixture(scope="module", params=[0, 1, 2, 3], ids=["direct_tc", "garner", "direct_int", "direct_tc_cvt"])
def c1(request):
    # N = 2^11, Q = P = 2^120 (the smallest workload), plus rotation keys; every reconstruction
    return make_pair(11, 120, 120, seed=11, rot_steps=(1, 3, -1, 1 << 10), crt=request.param)


def _messages(P, count, log_scale=30):
    N = P.prm.N
    return [encode.encode(fs.unit_disk(P.g, N // 2), N, log_scale) for _ in range(count)]


def test_encrypt_decrypt_match_oracle(c1):
    P = c1
    msgs = _messages(P, 3)
    ct, octs = encrypt_both(P, msgs)
    assert ct_ints(ct) == octs
    dec = P.ctx.decrypt(ct).cpu().numpy().view(np.uint32)
    for i in range(3):
        assert bigint.from_limbs(dec[i], signed=True) == ckks.decrypt(P.s, octs[i], P.prm.logQ)


def test_mult_relin_and_rescale_match_oracle(c1):
    P = c1
    ca, oa = encrypt_both(P, _messages(P, 2))
    cb, ob = encrypt_both(P, _messages(P, 2))
    got = ct_ints(P.ctx.mult_relin(ca, cb))
    want = [ckks.mult(x, y, P.evk, 120, 120) for x, y in zip(oa, ob)]
    assert got == [tuple(w) for w in want]
    got_rs = ct_ints(P.ctx.mult_relin_rescale(ca, cb, 30))
    assert got_rs == [tuple(ckks.rescale(w, 30, 120)) for w in want]


@pytest.mark.parametrize("logQ", [120, 97, 64, 33])
def test_mult_uniform_ciphertexts_at_lower_levels(c1, logQ):
    """Full-range ciphertexts (uniform limbs) at ragged and exact levels, with zero and all-ones rows."""
    P = c1
    N = P.prm.N
    la = random_ct_limbs(P.g, 2, N, logQ)
    lb = random_ct_limbs(P.g, 2, N, logQ)
    top = logQ - 32 * (fs.limb_count(logQ) - 1)
    la[1, :, :, :] = 0xFFFFFFFF
    la[1, :, -1, :] &= np.uint32((1 << top) - 1) if top < 32 else np.uint32(0xFFFFFFFF)
    lb[1, 0] = 0
    ca, cb = _ct_from_limbs(P, la, logQ), _ct_from_limbs(P, lb, logQ)
    got = ct_ints(P.ctx.mult_relin(ca, cb))
    want = [ckks.mult(x, y, P.evk, logQ, 120) for x, y in zip(_oracle_ct(la), _oracle_ct(lb))]
    assert got == [tuple(w) for w in want]


def test_rotations_match_oracle(c1):
    P = c1
    ct, octs = encrypt_both(P, _messages(P, 2, 40))
    for step in (1, 3, -1, 1 << 10):
        got = ct_ints(P.ctx.rotate(ct, step))
        want = [ckks.rotate(o, step, P.rtk[step], P.prm.N, 120, 120) for o in octs]
        assert got == [tuple(w) for w in want], step


def test_limb_operations_match_oracle(c1):
    P = c1
    N = P.prm.N
    la = random_ct_limbs(P.g, 2, N, 120)
    lb = random_ct_limbs(P.g, 2, N, 120)
    ca, cb = _ct_from_limbs(P, la, 120), _ct_from_limbs(P, lb, 120)
    oa, ob = _oracle_ct(la), _oracle_ct(lb)
    ctx = P.ctx
    assert ct_ints(ctx.add(ca, cb)) == [ckks.add(x, y, 120) for x, y in zip(oa, ob)]
    assert ct_ints(ctx.sub(ca, cb)) == [ckks.sub(x, y, 120) for x, y in zip(oa, ob)]
    assert ct_ints(ctx.negate(ca)) == [ckks.negate(x, 120) for x in oa]
    for c in (-7, 12345, 1, -1):
        assert ct_ints(ctx.mult_const(ca, c)) == [ckks.mult_const(x, c, 120) for x in oa]
    for k in (1, 30, 32, 33, 64, 119):
        assert ct_ints(ctx.rescale(ca, k)) == [tuple(ckks.rescale(x, k, 120)) for x in oa], k
    for lq in (100, 96, 1):
        assert ct_ints(ctx.moddown(ca, lq)) == [tuple(ckks.moddown(x, lq)) for x in oa], lq


def test_decoded_product_accuracy_c1(c1):
    """Decode(Dec(RS(Mult))) within 2^-10 of the FP64 slot product at scale 2^30 (GPU ciphertexts)."""
    P = c1
    N = P.prm.N
    z1, z2 = fs.unit_disk(P.g, N // 2), fs.unit_disk(P.g, N // 2)
    ca, _ = encrypt_both(P, [encode.encode(z1, N, 30)])
    cb, _ = encrypt_both(P, [encode.encode(z2, N, 30)])
    out = P.ctx.mult_relin_rescale(ca, cb, 30)
    dec = bigint.from_limbs(P.ctx.decrypt(out).cpu().numpy().view(np.uint32)[0], signed=True)
    z = encode.decode(dec, N, 30, N // 2)
    assert np.abs(z - z1 * z2).max() <= 2.0 ** -10 * max(1.0, np.abs(z1 * z2).max())


@pytest.mark.parametrize("crt", [0, 1, 2, 3], ids=["direct_tc", "garner", "direct_int", "direct_tc_cvt"])
def test_two_pass_ring_mid_size(crt):
    """N = 2^14 (two-pass NTT), logQ = logP = 438, a batch of two: mult+relin+rescale and a rotation."""
    P = make_pair(14, 438, 438, seed=14, rot_steps=(5,), crt=crt)
    N = P.prm.N
    la = random_ct_limbs(P.g, 2, N, 438)
    lb = random_ct_limbs(P.g, 2, N, 438)
    ca, cb = _ct_from_limbs(P, la, 438), _ct_from_limbs(P, lb, 438)
    got = ct_ints(P.ctx.mult_relin_rescale(ca, cb, 40))
    want = [tuple(ckks.rescale(ckks.mult(x, y, P.evk, 438, 438), 40, 438)) for x, y in zip(_oracle_ct(la), _oracle_ct(lb))]
    assert got == want
    got = ct_ints(P.ctx.rotate(ca, 5))
    assert got[0] == tuple(ckks.rotate(_oracle_ct(la)[0], 5, P.rtk[5], N, 438, 438))
    P.ctx.close()


@pytest.mark.slow
def test_full_size_pair_every_limb():
    """N = 2^16, logQ = logP = 1200, scale 2^40: one pair, every limb compared with the oracle."""
    import paper_2607_05920_gb300 as fhe

    P = make_pair(16, 1200, 1200, seed=16)
    N = P.prm.N
    la = random_ct_limbs(P.g, 1, N, 1200)
    lb = random_ct_limbs(P.g, 1, N, 1200)
    ca, cb = _ct_from_limbs(P, la, 1200), _ct_from_limbs(P, lb, 1200)
    got = ct_ints(P.ctx.mult_relin_rescale(ca, cb, 40))
    want = tuple(ckks.rescale(ckks.mult(_oracle_ct(la)[0], _oracle_ct(lb)[0], P.evk, 1200, 1200), 40, 1200))
    assert got[0] == want
    P.ctx.close()
    # the Garner and integer-pipe reconstructions give the same ciphertext from the same keys
    for mode in (fhe.FHE_CRT_GARNER, fhe.FHE_CRT_DIRECT_INT, fhe.FHE_CRT_DIRECT_CVT):
        Pg = make_pair(16, 1200, 1200, seed=16, crt=mode)
        assert ct_ints(Pg.ctx.mult_relin_rescale(ca, cb, 40))[0] == want
        Pg.ctx.close()


@pytest.mark.slow
def test_bench_configuration_sampled_pairs_match_the_oracle():
    """The benchmark's launch configuration (N = 2^16, logQ = logP = 1200, 64 pairs in one call):
    two pairs sampled from the batch, every limb compared with the oracle."""
    P = make_pair(16, 1200, 1200, seed=64)
    N = P.prm.N
    la = random_ct_limbs(P.g, 64, N, 1200)
    lb = random_ct_limbs(P.g, 64, N, 1200)
    out = P.ctx.mult_relin_rescale(_ct_from_limbs(P, la, 1200), _ct_from_limbs(P, lb, 1200), 40)
    host = out.data.cpu().numpy().view(np.uint32)
    P.ctx.close()
    for c in (0, 45):  # a pair from the first tiles and one from the persistent CTAs' later sweeps
        got = tuple(bigint.from_limbs(host[c, p]) for p in range(2))
        want = tuple(ckks.rescale(ckks.mult(_oracle_ct(la[c:c + 1])[0], _oracle_ct(lb[c:c + 1])[0], P.evk, 1200, 1200),
                                  40, 1200))
        assert got == want, c


@pytest.mark.slow
def test_full_size_batch_tensor_core_crt_equals_integer_crt():
    """N = 2^16, logQ = logP = 1200, cnum 8: the tensor-core and integer reconstructions agree on every limb."""
    import paper_2607_05920_gb300 as fhe
    import torch

    outs = []
    for mode in (fhe.FHE_CRT_DIRECT, fhe.FHE_CRT_DIRECT_INT, fhe.FHE_CRT_DIRECT_CVT):
        P = make_pair(16, 1200, 1200, seed=17, crt=mode)
        g = fs.rng(170)
        la = random_ct_limbs(g, 8, P.prm.N, 1200)
        lb = random_ct_limbs(g, 8, P.prm.N, 1200)
        out = P.ctx.mult_relin_rescale(_ct_from_limbs(P, la, 1200), _ct_from_limbs(P, lb, 1200), 40)
        outs.append(out.data.cpu())
        P.ctx.close()
    assert torch.equal(outs[0], outs[1])
    assert torch.equal(outs[0], outs[2])
