"""The rest of the HEAAN operation set against the oracle (needs a GB300).

imult (x X^(N/2)), multconstvec (ciphertext x plaintext polynomial, pairwise
and broadcast), addconst with one constant per ciphertext, and the broadcast
mode of mult / add / sub (one ciphertext applied across a CipherTensor).
Every limb must equal the oracle's.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, ckks, encode

from fhe_setup import ct_ints, make_pair, random_ct_limbs, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p11():
    P = make_pair(11, 120, 120, seed=411)
    yield P
    P.ctx.close()


def _ct(fhe, limbs, logQ, scale=0.0):
    return fhe.Ciphertext(to_dev(limbs), logQ, log_scale=scale)


def _o(limbs):
    return [tuple(bigint.from_limbs(limbs[c, p]) for p in range(2)) for c in range(limbs.shape[0])]


def test_imult_matches_oracle(p11):
    import paper_2607_05920_gb300 as fhe

    la = random_ct_limbs(p11.g, 3, 2048, 97)
    out = p11.ctx.imult(_ct(fhe, la, 97, 40))
    assert out.log_scale == 40
    assert ct_ints(out) == [ckks.imult(o, 2048, 97) for o in _o(la)]


@pytest.mark.parametrize("pt_cnum", [3, 1], ids=["pairwise", "broadcast"])
def test_mult_plain_matches_oracle(p11, pt_cnum):
    import paper_2607_05920_gb300 as fhe

    N, logQ = 2048, 120
    la = random_ct_limbs(p11.g, 3, N, logQ)
    msgs = [[int(x) for x in fs.small_signed(p11.g, (), N, 35)] for _ in range(pt_cnum)]
    mask = (1 << logQ) - 1
    pt = np.stack([bigint.to_limbs([x & mask for x in m], fhe.limbs(logQ)) for m in msgs])
    out = p11.ctx.mult_plain(_ct(fhe, la, logQ, 40), to_dev(pt), pt_log_scale=30)
    assert out.log_scale == 70
    want = [ckks.mult_plain(o, msgs[c if pt_cnum > 1 else 0], logQ) for c, o in enumerate(_o(la))]
    assert ct_ints(out) == [tuple(w) for w in want]


def test_add_const_vec_matches_oracle(p11):
    import torch

    import paper_2607_05920_gb300 as fhe

    la = random_ct_limbs(p11.g, 4, 2048, 120)
    vals = [5, -7, (1 << 62) - 1, -(1 << 40)]
    out = p11.ctx.add_const_vec(_ct(fhe, la, 120), torch.tensor(vals, dtype=torch.int64, device="cuda"), 30)
    assert ct_ints(out) == [tuple(ckks.add_const(o, v << 30, 120)) for o, v in zip(_o(la), vals)]


def test_broadcast_mult_add_sub_match_oracle(p11):
    import paper_2607_05920_gb300 as fhe

    N, logQ = 2048, 120
    la = random_ct_limbs(p11.g, 3, N, logQ)
    lb = random_ct_limbs(p11.g, 1, N, logQ)
    ca, cb = _ct(fhe, la, logQ), _ct(fhe, lb, logQ)
    ob = _o(lb)[0]
    got = ct_ints(p11.ctx.mult_relin_rescale(ca, cb, 30))
    assert got == [tuple(ckks.rescale(ckks.mult(o, ob, p11.evk, logQ, 120), 30, logQ)) for o in _o(la)]
    assert ct_ints(p11.ctx.add(ca, cb)) == [ckks.add(o, ob, logQ) for o in _o(la)]
    assert ct_ints(p11.ctx.sub(ca, cb)) == [ckks.sub(o, ob, logQ) for o in _o(la)]


def test_mult_plain_decodes_to_the_slot_product():
    import paper_2607_05920_gb300 as fhe

    P = make_pair(12, 200, 200, seed=412)
    N, n = P.prm.N, P.prm.N // 2
    z1, z2 = fs.unit_disk(P.g, n), fs.unit_disk(P.g, n)
    from fhe_setup import encrypt_both

    ct, _ = encrypt_both(P, [encode.encode(z1, N, 40)])
    ct.log_scale = 40
    m2 = encode.encode(z2, N, 30)
    pt = to_dev(bigint.to_limbs([x & ((1 << 200) - 1) for x in m2], fhe.limbs(200))[None])
    out = P.ctx.rescale(P.ctx.mult_plain(ct, pt, 30), 30)
    assert out.log_scale == 40
    dec = bigint.from_limbs(P.ctx.decrypt(out).cpu().numpy().view(np.uint32)[0], signed=True)
    assert np.abs(encode.decode(dec, N, 40, n) - z1 * z2).max() <= 2.0 ** -20
    P.ctx.close()


def test_empty_out_of_range_and_degenerate_inputs(p11):
    """Edge cases through the C ABI: an empty batch (cnum 0) and a level above the context's top are
    rejected before anything is enqueued, leaving the output untouched; a product of two zero
    ciphertexts is the zero ciphertext (relinearisation and rescale of zero, rounding included)."""
    import ctypes

    import torch

    import paper_2607_05920_gb300 as fhe

    ctx = p11.ctx
    N = 1 << 11
    a = _ct(fhe, random_ct_limbs(fs.rng(7), 2, N, 120), 120)
    out = ctx.empty_ct(2, 90)
    out.data.fill_(-1)
    before = out.data.clone()
    ws = ctx.workspace(fhe.FHE_OP_MULT, 120, 2)
    empty = fhe.FheCt(a.data.data_ptr(), 0, 120, 0, 0.0)
    eo = fhe.FheCt(out.data.data_ptr(), 0, 90, 0, 0.0)
    rc = fhe.lib.fhe_mult_relin_rescale(ctx.handle, ctypes.byref(empty), ctypes.byref(empty), 30, ctypes.byref(eo),
                                        ws.data_ptr(), ws.numel(), None)
    assert rc == fhe.FHE_EINVAL
    assert fhe.lib.fhe_rescale(ctx.handle, ctypes.byref(empty), 30, ctypes.byref(eo), None) == fhe.FHE_EINVAL
    assert fhe.lib.fhe_add(ctx.handle, ctypes.byref(empty), ctypes.byref(empty), ctypes.byref(empty), None) == \
        fhe.FHE_EINVAL
    high = fhe.FheCt(a.data.data_ptr(), 2, 121, 0, 0.0)  # above the context's logQ = 120
    rc = fhe.lib.fhe_mult_relin_rescale(ctx.handle, ctypes.byref(high), ctypes.byref(high), 31, ctypes.byref(
        fhe.FheCt(out.data.data_ptr(), 2, 90, 0, 0.0)), ws.data_ptr(), ws.numel(), None)
    assert rc in (fhe.FHE_EINVAL, fhe.FHE_ELEVEL)
    torch.cuda.synchronize()
    assert torch.equal(out.data, before)
    zero = _ct(fhe, np.zeros((2, 2, 4, N), dtype=np.uint32), 120)
    res = ctx.empty_ct(2, 90)
    fhe.fhe_mult_relin_rescale(ctx, zero, zero, 30, res)
    torch.cuda.synchronize()
    assert int(res.data.abs().sum()) == 0
