"""Hoisted rotations and conjugation against the oracle (needs a GB300).

fhe_rotate_hoisted lifts and transforms the key-switch input once and applies
each automorphism as a permutation of the transform; every output must equal
fhe_rotate of the same step and the oracle's rotation, bit for bit.  Both
ring-size paths run: N = 2^11 (one-CTA transforms, separate key products) and
N = 2^14 (the fused row pass with the row gather).
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, ckks, encode

from fhe_setup import ct_ints, encrypt_both, make_pair, random_ct_limbs, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("logN,logQ", [(11, 120), (14, 438)])
def test_hoisted_rotations_equal_single_rotations_and_oracle(logN, logQ):
    import torch

    import paper_2607_05920_gb300 as fhe

    N = 1 << logN
    steps = [1, -1, 5, N // 2, 3, 1 << (logN - 3)]
    P = make_pair(logN, logQ, logQ, seed=300 + logN, rot_steps=sorted(set(steps)), conj=True)
    la = random_ct_limbs(P.g, 3, N, logQ)
    la[2, 1, :, :] = 0  # a zero a-polynomial and one with its top bit set everywhere (negative centred value)
    la[2, 1, fhe.limbs(logQ) - 1, :] = np.uint32(1 << ((logQ - 1) % 32))
    ct = fhe.Ciphertext(to_dev(la), logQ, log_scale=40)
    outs = P.ctx.rotate_hoisted(ct, steps)
    oct_ = [tuple(bigint.from_limbs(la[c, p]) for p in range(2)) for c in range(3)]
    for step, out in zip(steps, outs):
        assert out.log_scale == 40
        single = P.ctx.rotate(ct, step)
        assert torch.equal(single.data, out.data), step
        got = ct_ints(out)
        for c in (0, 2):
            assert got[c] == tuple(ckks.rotate(oct_[c], step, P.rtk[step], N, logQ, logQ)), (step, c)
    got = ct_ints(P.ctx.conjugate(ct))
    for c in range(3):
        assert got[c] == tuple(ckks.conjugate(oct_[c], P.ck, N, logQ, logQ)), c
    P.ctx.close()


def test_conjugate_and_rotations_decode():
    """Encrypted slots at scale 2^40: conjugation gives conj(z) and hoisted rotations give the shifted slots,
    within 2^-20."""
    P = make_pair(12, 200, 200, seed=312, rot_steps=(1, 2, 4, 8), conj=True)
    N, n = P.prm.N, P.prm.N // 2
    z = fs.unit_disk(P.g, n)
    ct, _ = encrypt_both(P, [encode.encode(z, N, 40)])

    def dec(c):
        return encode.decode(bigint.from_limbs(P.ctx.decrypt(c).cpu().numpy().view(np.uint32)[0], signed=True), N, 40, n)

    assert np.abs(dec(P.ctx.conjugate(ct)) - np.conj(z)).max() <= 2.0 ** -20
    for step, out in zip((1, 2, 4, 8), P.ctx.rotate_hoisted(ct, (1, 2, 4, 8))):
        assert np.abs(dec(out) - np.roll(z, -step)).max() <= 2.0 ** -20, step
    P.ctx.close()


def test_rotate_argument_errors():
    import paper_2607_05920_gb300 as fhe

    P = make_pair(11, 120, 120, seed=313, rot_steps=(1,))
    ct = fhe.Ciphertext(to_dev(random_ct_limbs(P.g, 1, 2048, 120)), 120)
    with pytest.raises(fhe.FheError) as e:
        P.ctx.rotate(ct, 2)  # no key
    assert e.value.code == fhe.FHE_ENOKEY
    with pytest.raises(fhe.FheError) as e:
        P.ctx.conjugate(ct)  # no conjugation key
    assert e.value.code == fhe.FHE_ENOKEY
    out = P.ctx.empty_ct(1, 120)
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_rotate_hoisted(P.ctx, ct, [1, 1], [out, out])  # aliasing outputs
    assert e.value.code == fhe.FHE_EINVAL
    P.ctx.close()
