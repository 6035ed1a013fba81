"""GPU path vs the oracle at the workloads' own sizes (needs a GB300).

* uneven batches at the large ring sizes of the batched workload (N = 2^13 and
  2^16, items at three levels up to logQ = 1200 in one ragged call: the
  two-pass NTT together with the per-item-modulus epilogue);
* the serving width N = 2^16, logQ = logP = 1550 (about 156 key-switch primes,
  97 output limbs: the streamed tensor-core reconstruction at its widest);
* the sparse-secret workload N = 2^15, logQ = logP = 880 with a Hamming-weight
  64 secret: one pair and rotations by 2^0, 2^7 and 2^14 slots (2^14 is the
  identity automorphism at this ring size);
* fhe_add_const against the oracle's addconst;
* the stated CKKS accuracy: decoded slots of a product at scale 2^40 within
  2^-20 (relative to max(1, |z1 z2|)) of the FP64 product.

Oracle products at N = 2^15 and 2^16 take seconds each, so these tests compare
one or a few ciphertexts, every limb of each.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, ckks, encode

from fhe_setup import ct_ints, encrypt_both, make_pair, random_ct_limbs, to_dev

pytestmark = pytest.mark.gpu


def _oracle_item(host, c):
    return tuple(bigint.from_limbs(host[c, p]) for p in range(2))


def _ragged_case(logN, levels, seed, k=40):
    import torch

    import paper_2607_05920_gb300 as fhe

    P = make_pair(logN, 1200, 1200, seed=seed)
    N = P.prm.N
    g = fs.rng(seed + 1)
    L_pad = fhe.limbs(max(levels))
    n = len(levels)
    a = np.zeros((n, 2, L_pad, N), dtype=np.uint32)
    b = np.zeros_like(a)
    for i, lq in enumerate(levels):
        a[i, :, :fhe.limbs(lq)] = fs.uniform_limbs(g, (2,), N, lq)
        b[i, :, :fhe.limbs(lq)] = fs.uniform_limbs(g, (2,), N, lq)
    A, B = to_dev(a), to_dev(b)
    O = torch.empty_like(A)
    bits = torch.tensor(levels, dtype=torch.int32, device=A.device)
    fhe.fhe_mult_relin_rescale_ragged(P.ctx, A, B, O, bits, max(levels), k)
    host = O.cpu().numpy().view(np.uint32)
    for i, lq in enumerate(levels):
        L_out = fhe.limbs(lq - k)
        assert not host[i, :, L_out:].any(), f"item {i}: limbs above its level are not zero"
        # the same pair through the plain call at its own level
        ca = fhe.Ciphertext(to_dev(a[i:i + 1, :, :fhe.limbs(lq)]), lq)
        cb = fhe.Ciphertext(to_dev(b[i:i + 1, :, :fhe.limbs(lq)]), lq)
        per_op = P.ctx.mult_relin_rescale(ca, cb, k).data.cpu().numpy().view(np.uint32)
        assert np.array_equal(per_op[0], host[i, :, :L_out]), f"item {i} differs from the per-op call"
        want = ckks.rescale(ckks.mult(_oracle_item(a[:, :, :fhe.limbs(lq)], i), _oracle_item(b[:, :, :fhe.limbs(lq)], i),
                                      P.evk, lq, 1200), k, lq)
        assert _oracle_item(host[:, :, :L_out], i) == tuple(want), f"item {i} (logQ {lq}) differs from the oracle"
    P.ctx.close()


def test_ragged_batch_at_n_2_13_three_levels():
    _ragged_case(13, [1200, 437, 201], seed=131)


@pytest.mark.slow
def test_ragged_batch_at_n_2_16_three_levels():
    _ragged_case(16, [777, 1200, 230], seed=161)


@pytest.mark.slow
def test_serving_width_mult_and_rotation_match_oracle():
    """N = 2^16, logQ = logP = 1550: one HMult+relin+rescale and one rotation, every limb."""
    P = make_pair(16, 1550, 1550, seed=155, rot_steps=(4,))
    N = P.prm.N
    la = random_ct_limbs(P.g, 1, N, 1550)
    lb = random_ct_limbs(P.g, 1, N, 1550)
    import paper_2607_05920_gb300 as fhe

    ca, cb = fhe.Ciphertext(to_dev(la), 1550), fhe.Ciphertext(to_dev(lb), 1550)
    got = ct_ints(P.ctx.mult_relin_rescale(ca, cb, 40))[0]
    oa, ob = _oracle_item(la, 0), _oracle_item(lb, 0)
    assert got == tuple(ckks.rescale(ckks.mult(oa, ob, P.evk, 1550, 1550), 40, 1550))
    got = ct_ints(P.ctx.rotate(ca, 4))[0]
    assert got == tuple(ckks.rotate(oa, 4, P.rtk[4], N, 1550, 1550))
    P.ctx.close()


@pytest.mark.slow
def test_sparse_secret_workload_pair_and_rotations():
    """N = 2^15, logQ = logP = 880, Hamming-weight-64 secret, scale 2^40: a product and rotations by
    2^0, 2^7, 2^14 slots match the oracle bit for bit and decode within the stated accuracy."""
    steps = (1, 1 << 7, 1 << 14)
    P = make_pair(15, 880, 880, seed=215, hwt=64, rot_steps=steps)
    N, n = P.prm.N, P.prm.N // 2
    assert sum(1 for x in P.s if x != 0) == 64
    z1, z2 = fs.unit_disk(P.g, n), fs.unit_disk(P.g, n)
    ca, oa = encrypt_both(P, [encode.encode(z1, N, 40)])
    cb, ob = encrypt_both(P, [encode.encode(z2, N, 40)])
    assert ct_ints(ca) == oa
    out = P.ctx.mult_relin_rescale(ca, cb, 40)
    want = ckks.rescale(ckks.mult(oa[0], ob[0], P.evk, 880, 880), 40, 880)
    assert ct_ints(out)[0] == tuple(want)
    dec = bigint.from_limbs(P.ctx.decrypt(out).cpu().numpy().view(np.uint32)[0], signed=True)
    z = encode.decode(dec, N, 40, n)
    assert np.abs(z - z1 * z2).max() <= 2.0 ** -20 * max(1.0, np.abs(z1 * z2).max())
    import torch

    hoisted = P.ctx.rotate_hoisted(ca, steps)
    for step, h in zip(steps, hoisted):
        got = P.ctx.rotate(ca, step)
        assert torch.equal(h.data, got.data), step
        assert ct_ints(got)[0] == tuple(ckks.rotate(oa[0], step, P.rtk[step], N, 880, 880)), step
        dec = bigint.from_limbs(P.ctx.decrypt(got).cpu().numpy().view(np.uint32)[0], signed=True)
        assert np.abs(encode.decode(dec, N, 40, n) - np.roll(z1, -step)).max() <= 2.0 ** -20, step
    P.ctx.close()


def test_add_const_matches_oracle():
    import paper_2607_05920_gb300 as fhe

    P = make_pair(11, 120, 120, seed=77)
    N = P.prm.N
    la = random_ct_limbs(P.g, 2, N, 97)
    la[1, 0, :, 0] = 0xFFFFFFFF  # a carry through every limb
    la[1, 0, -1, 0] &= 1
    ct = fhe.Ciphertext(to_dev(la), 97)
    for value, shift in ((12345, 0), (-1, 0), (-(1 << 40) + 3, 30), ((1 << 62) - 1, 34), (7, 96)):
        out = P.ctx.empty_ct(2, 97)
        fhe.fhe_add_const(P.ctx, ct, value, shift, out)
        want = [ckks.add_const(_oracle_item(la, c), value << shift, 97) for c in range(2)]
        assert ct_ints(out) == [tuple(w) for w in want], (value, shift)
    P.ctx.close()


def test_decoded_product_accuracy_at_scale_2_40():
    """Decode(Dec(RS_40(Mult(Enc z1, Enc z2)))) within 2^-20 max(1, |z1 z2|) of the FP64 product
    (N = 2^12, logQ = logP = 200, scale 2^40, slots uniform in the unit disk)."""
    P = make_pair(12, 200, 200, seed=240)
    N, n = P.prm.N, P.prm.N // 2
    z1, z2 = fs.unit_disk(P.g, n), fs.unit_disk(P.g, n)
    ca, _ = encrypt_both(P, [encode.encode(z1, N, 40)])
    cb, _ = encrypt_both(P, [encode.encode(z2, N, 40)])
    out = P.ctx.mult_relin_rescale(ca, cb, 40)
    dec = bigint.from_limbs(P.ctx.decrypt(out).cpu().numpy().view(np.uint32)[0], signed=True)
    z = encode.decode(dec, N, 40, n)
    err = np.abs(z - z1 * z2).max()
    assert err <= 2.0 ** -20 * max(1.0, np.abs(z1 * z2).max()), err
    P.ctx.close()
