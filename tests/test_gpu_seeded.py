"""Seeded key generation and encryption against the oracle (needs a GB300).

fhe_keygen(seed) and fhe_encrypt(seed) draw every random polynomial inside
the library (Philox4x32-10 on the host for keys, in a kernel for the
randomness of encryption).  The oracle draws the same polynomials with its
own implementation of the same generator (oracle/sampler.py) and builds the
keys and ciphertexts from its scheme definitions; every limb must agree.
Also: the scale bookkeeping of fhe_ct.log_scale.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bgv, bigint, ckks, encode
from oracle import sampler as S

from fhe_setup import ct_ints, to_dev

pytestmark = pytest.mark.gpu


def _oracle_keys(prm, seed, hwt=0, steps=()):
    N = prm.N
    s = S.sparse_ternary(seed, S.TAG_SECRET, 0, N, hwt) if hwt else S.ternary(seed, S.TAG_SECRET, 0, N)
    si = [int(x) for x in s]
    pk = ckks.public_key(prm, si, bigint.from_limbs(S.uniform_limbs(seed, S.TAG_PK_A, 0, N, prm.logQ)),
                         [int(x) for x in S.gaussian(seed, S.TAG_PK_E, 0, N)])
    evk = ckks.relin_key(prm, si, bigint.from_limbs(S.uniform_limbs(seed, S.TAG_EV_A, 0, N, prm.logQ + prm.logP)),
                         [int(x) for x in S.gaussian(seed, S.TAG_EV_E, 0, N)])
    rtk = {}
    for step in steps:
        g = ckks.galois_element(N, step)
        rtk[step] = ckks.rotation_key(prm, si, step, bigint.from_limbs(S.uniform_limbs(seed, S.TAG_SW_A, g, N,
                                                                                        prm.logQ + prm.logP)),
                                      [int(x) for x in S.gaussian(seed, S.TAG_SW_E, g, N)])
    return si, pk, evk, rtk


def _oracle_encrypt(prm, pk, msgs, seed, logQ):
    out = []
    for c, m in enumerate(msgs):
        v = [int(x) for x in S.ternary(seed, S.TAG_ENC_V, c, prm.N)]
        e0 = [int(x) for x in S.gaussian(seed, S.TAG_ENC_E0, c, prm.N)]
        e1 = [int(x) for x in S.gaussian(seed, S.TAG_ENC_E1, c, prm.N)]
        out.append(ckks.encrypt(prm, pk, m, v, e0, e1, logQ=logQ))
    return out


def _pt(fhe, msgs, logQ):
    mask = (1 << logQ) - 1
    return to_dev(np.stack([bigint.to_limbs([x & mask for x in m], fhe.limbs(logQ)) for m in msgs]))


@pytest.mark.parametrize("logN,logQ,hwt", [(11, 120, 0), (12, 200, 64)])
def test_seeded_keys_and_encryption_match_oracle(logN, logQ, hwt):
    import paper_2607_05920_gb300 as fhe

    seed_k, seed_e = 0x1234_5678_9ABC_DEF0 + logN, 77 + logN
    steps = (1, -3)
    ctx = fhe.Context(logN, logQ, logQ, hamming_weight=hwt)
    ctx.keygen(seed_k, rot_steps=steps)
    prm = ckks.CkksParams(logN, logQ, logQ)
    s, pk, evk, rtk = _oracle_keys(prm, seed_k, hwt, steps)
    assert hwt == 0 or sum(1 for x in s if x) == hwt
    g = fs.rng(logN)
    msgs = [encode.encode(fs.unit_disk(g, prm.N // 2), prm.N, 40) for _ in range(3)]
    ct = ctx.encrypt(_pt(fhe, msgs, logQ), seed_e, log_scale=40)
    octs = _oracle_encrypt(prm, pk, msgs, seed_e, logQ)
    assert ct_ints(ct) == octs
    # the resident secret decrypts as the oracle's secret does
    dec = ctx.decrypt(ct).cpu().numpy().view(np.uint32)
    assert bigint.from_limbs(dec[1], signed=True) == ckks.decrypt(s, octs[1], logQ)
    # relinearisation and rotation keys
    out = ctx.mult_relin_rescale(ct, ct, 40)
    assert ct_ints(out) == [tuple(ckks.rescale(ckks.mult(o, o, evk, logQ, logQ), 40, logQ)) for o in octs]
    for step in steps:
        assert ct_ints(ctx.rotate(ct, step)) == [tuple(ckks.rotate(o, step, rtk[step], prm.N, logQ, logQ))
                                                 for o in octs]
    ctx.close()


def test_seeded_encryption_is_a_function_of_the_seed():
    import torch

    import paper_2607_05920_gb300 as fhe

    ctx = fhe.Context(11, 120, 120)
    ctx.keygen(5)
    pt = to_dev(np.zeros((2, 4, 2048), dtype=np.uint32))
    a, b, c = ctx.encrypt(pt, 9), ctx.encrypt(pt, 9), ctx.encrypt(pt, 10)
    assert torch.equal(a.data, b.data) and not torch.equal(a.data, c.data)
    # the two ciphertexts of one call differ (tag1 = the index in the batch)
    assert not torch.equal(a.data[0], a.data[1])
    ctx.close()


def test_seeded_bgv_keys_match_oracle_and_decrypt_exactly():
    import paper_2607_05920_gb300 as fhe

    t, levels, logN = 65537, 8, 10
    q0, r = bgv.chain_moduli(t, 54, 48)
    logQ = (q0 * r ** levels).bit_length()
    prm = bgv.BgvParams(logN, t, q0, r, levels, logQ)
    N = prm.N
    ctx = fhe.Context(logN, logQ, logQ, scheme=fhe.FHE_SCHEME_BGV, t=t, bgv_q0=q0, bgv_r=r, bgv_levels=levels)
    seed = 4242
    ctx.keygen(seed)
    Lq, Lpq = fhe.limbs(logQ), fhe.limbs(2 * logQ)
    si = [int(x) for x in S.ternary(seed, S.TAG_SECRET, 0, N)]
    Q, PQ = prm.Qtop, prm.P * prm.Qtop
    pk = bgv.public_key(prm, si, [x % Q for x in bigint.from_limbs(S.uniform_limbs(seed, S.TAG_PK_A, 0, N, 32 * Lq))],
                        [int(x) for x in S.gaussian(seed, S.TAG_PK_E, 0, N)])
    evk = bgv.relin_key(prm, si,
                        [x % PQ for x in bigint.from_limbs(S.uniform_limbs(seed, S.TAG_EV_A, 0, N, 32 * Lpq))],
                        [int(x) for x in S.gaussian(seed, S.TAG_EV_E, 0, N)])
    m = fs.uniform_mod_t(fs.rng(3), (1,), N, t)
    pt = np.zeros((1, Lq, N), dtype=np.uint32)
    pt[:, 0, :] = m.astype(np.uint32)
    seed_e = 99
    ct = ctx.encrypt(to_dev(pt), seed_e)
    o = bgv.encrypt(prm, pk, [int(x) for x in m[0]], [int(x) for x in S.ternary(seed_e, S.TAG_ENC_V, 0, N)],
                    [int(x) for x in S.gaussian(seed_e, S.TAG_ENC_E0, 0, N)],
                    [int(x) for x in S.gaussian(seed_e, S.TAG_ENC_E1, 0, N)])
    assert ct_ints(ct)[0] == tuple(o)
    sq = ctx.mult_relin(ct, ct)
    assert ct_ints(sq)[0] == tuple(bgv.mult(prm, o, o, evk, levels))
    dec = ctx.decrypt(sq).cpu().numpy()[0]
    assert [int(x) for x in dec] == bgv.plaintext_power([int(x) for x in m[0]], 1, N, t)
    ctx.close()


def test_log_scale_bookkeeping():
    import paper_2607_05920_gb300 as fhe

    ctx = fhe.Context(11, 120, 120)
    ctx.keygen(1)
    pt = to_dev(np.zeros((1, 4, 2048), dtype=np.uint32))
    a = ctx.encrypt(pt, 2, log_scale=30)
    b = ctx.encrypt(pt, 3, log_scale=30)
    assert a.log_scale == 30
    assert ctx.mult_relin(a, b).log_scale == 60
    ab = ctx.mult_relin_rescale(a, b, 30)
    assert ab.log_scale == 30 and ab.logQ == 90
    assert ctx.rescale(ctx.mult_relin(a, b), 20).log_scale == 40
    assert ctx.moddown(a, 90).log_scale == 30
    assert ctx.add(a, b).log_scale == 30 and ctx.negate(a).log_scale == 30
    assert ctx.mult_const(a, 3).log_scale == 30
    c = ctx.encrypt(pt, 4, log_scale=31)
    with pytest.raises(fhe.FheError) as err:
        ctx.add(a, c)
    assert err.value.code == fhe.FHE_ELEVEL
    ctx.close()
