"""BGV on the GPU vs the oracle (needs a GB300).

Bit-exact ciphertexts against oracle/bgv.py after every multiplication and
modulus switch of a squaring chain, and exact decryption mod t, at a small
ring with the full-size chain (q0 ~ 2^54, r ~ 2^48, 8 levels, logQ = 438,
P = 2^438) and at the N = 2^14, t = 65537 workload size on a batch.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bgv, bigint

from fhe_setup import to_dev

pytestmark = pytest.mark.gpu

T = 65537


def _setup(logN, levels, seed, cnum):
    import paper_2607_05920_gb300 as fhe

    q0, r = bgv.chain_moduli(T, 54, 48)
    logQ = (q0 * r ** levels).bit_length()
    logP = logQ
    prm = bgv.BgvParams(logN, T, q0, r, levels, logP)
    N = prm.N
    g = fs.rng(seed)
    s = fs.ternary(g, (), N)
    a_pk = fs.uniform_limbs(g, (), N, logQ)
    e_pk = fs.gaussian(g, (), N)
    a_ev = fs.uniform_limbs(g, (), N, logQ + logP)
    e_ev = fs.gaussian(g, (), N)
    ctx = fhe.Context(logN, logQ, logP, scheme=fhe.FHE_SCHEME_BGV, t=T, bgv_q0=q0, bgv_r=r, bgv_levels=levels)
    ctx.keygen_inject(s, a_pk, e_pk, a_ev, e_ev)
    si = [int(x) for x in s]
    Q, PQ = prm.Qtop, prm.P * prm.Qtop
    pk = bgv.public_key(prm, si, [x % Q for x in bigint.from_limbs(a_pk)], [int(x) for x in e_pk])
    evk = bgv.relin_key(prm, si, [x % PQ for x in bigint.from_limbs(a_ev)], [int(x) for x in e_ev])
    m = fs.uniform_mod_t(g, (cnum,), N, T)
    v = fs.ternary(g, (cnum,), N)
    e0 = fs.gaussian(g, (cnum,), N)
    e1 = fs.gaussian(g, (cnum,), N)
    L = fhe.limbs(logQ)
    pt = np.zeros((cnum, L, N), dtype=np.uint32)
    pt[:, 0, :] = m.astype(np.uint32)
    ct = ctx.encrypt_inject(to_dev(pt), to_dev(v), to_dev(e0), to_dev(e1))
    return fhe, ctx, prm, si, pk, evk, m, v, e0, e1, ct


def _ints(ct, c):
    host = ct.data.cpu().numpy().view(np.uint32)
    return tuple(bigint.from_limbs(host[c, p]) for p in range(2))


def test_bgv_chain_bit_exact_small_ring():
    """N = 2^10, full chain: every ciphertext equals the oracle's, every decryption is m^(2^k) mod t."""
    fhe, ctx, prm, s, pk, evk, m, v, e0, e1, ct = _setup(10, 8, 31, 1)
    o = bgv.encrypt(prm, pk, [int(x) for x in m[0]], [int(x) for x in v[0]], [int(x) for x in e0[0]],
                    [int(x) for x in e1[0]])
    assert _ints(ct, 0) == o
    level = prm.levels
    for k in range(1, prm.levels + 1):
        ct = ctx.mult_relin(ct, ct)
        o = bgv.mult(prm, o, o, evk, level)
        assert _ints(ct, 0) == o, f"mult {k}"
        ct = ctx.mod_switch(ct)
        o = bgv.mod_switch(prm, o, level)
        level -= 1
        assert _ints(ct, 0) == o, f"modswitch {k}"
        dec = ctx.decrypt(ct).cpu().numpy().view(np.uint32)[0]
        assert [int(x) for x in dec] == bgv.plaintext_power([int(x) for x in m[0]], k, prm.N, T)
    ctx.close()


def test_bgv_add_sub_negate_match_oracle():
    fhe, ctx, prm, s, pk, evk, m, v, e0, e1, ct = _setup(8, 3, 32, 2)
    a = fhe.Ciphertext(ct.data[:1].clone(), ct.logQ, ct.level)
    b = fhe.Ciphertext(ct.data[1:].clone(), ct.logQ, ct.level)
    Q = prm.Qtop
    oa, ob = _ints(a, 0), _ints(b, 0)
    assert _ints(ctx.add(a, b), 0) == tuple([(x + y) % Q for x, y in zip(pa, pb)] for pa, pb in zip(oa, ob))
    assert _ints(ctx.sub(a, b), 0) == tuple([(x - y) % Q for x, y in zip(pa, pb)] for pa, pb in zip(oa, ob))
    assert _ints(ctx.negate(a), 0) == tuple([(-x) % Q for x in pa] for pa in oa)
    ctx.close()


@pytest.mark.slow
def test_bgv_workload_size_chain():
    """N = 2^14, t = 65537, logQ = 438, a batch of 16 through the depth-8 chain; sampled oracle checks."""
    fhe, ctx, prm, s, pk, evk, m, v, e0, e1, ct = _setup(14, 8, 33, 16)
    o = bgv.encrypt(prm, pk, [int(x) for x in m[0]], [int(x) for x in v[0]], [int(x) for x in e0[0]],
                    [int(x) for x in e1[0]])
    assert _ints(ct, 0) == o
    ct = ctx.mult_relin(ct, ct)
    o = bgv.mult(prm, o, o, evk, prm.levels)
    assert _ints(ct, 0) == o
    ct = ctx.mod_switch(ct)
    assert _ints(ct, 0) == bgv.mod_switch(prm, o, prm.levels)
    for k in range(2, prm.levels + 1):
        ct = ctx.mod_switch(ctx.mult_relin(ct, ct))
    dec = ctx.decrypt(ct).cpu().numpy().view(np.uint32)
    for c in (0, 7, 15):
        assert [int(x) for x in dec[c]] == bgv.plaintext_power([int(x) for x in m[c]], prm.levels, prm.N, T)
    ctx.close()
