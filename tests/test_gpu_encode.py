"""Plaintext encoding on the GPU against the oracle (needs a GB300).

CKKS: fhe_ckks_encode / fhe_ckks_decode (double-precision DFTs) against the
oracle's canonical-embedding encoder (numpy FFT).  Encoded coefficients may
differ by one where the exact value sits within rounding distance of a
half-integer; decoded slots agree to 1e-9.  End to end, GPU-encoded products
decode within the stated 2^-20.
BGV: slot encoding and decoding (the polynomial CRT mod t) bit for bit
against the oracle's direct sums, and slot-wise products through encryption.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bgv, bigint, encode

from fhe_setup import make_pair, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("logN", [11, 16])
def test_ckks_encode_decode_match_oracle(logN):
    import torch

    import paper_2607_05920_gb300 as fhe

    N, logQ = 1 << logN, 200
    ctx = fhe.Context(logN, logQ, logQ)
    g = fs.rng(600 + logN)
    z = np.stack([fs.unit_disk(g, N // 2) for _ in range(2)])
    pt = fhe.fhe_ckks_encode(ctx, torch.from_numpy(z).cuda(), 40, logQ).cpu().numpy().view(np.uint32)
    for c in range(2):
        got = bigint.from_limbs(pt[c], signed=False)
        got = [x - (1 << logQ) if x >= 1 << (logQ - 1) else x for x in got]
        want = encode.encode(z[c], N, 40)
        diff = np.abs(np.array(got, dtype=object) - np.array(want, dtype=object)).astype(np.int64)
        assert diff.max() <= 1 and (diff > 0).mean() < 1e-3
    # decode: signed plaintexts of encoded size, in two's complement over L limbs
    m = fs.small_signed(g, (2,), N, 45)
    limbs = np.stack([bigint.to_limbs([int(x) for x in m[c]], fhe.limbs(logQ)) for c in range(2)])
    zz = fhe.fhe_ckks_decode(ctx, to_dev(limbs), logQ, 40).cpu().numpy()
    for c in range(2):
        want = encode.decode([int(x) for x in m[c]], N, 40, N // 2)
        assert np.abs(zz[c] - want).max() < 1e-9
    ctx.close()


def test_gpu_encoded_product_decodes_within_bound():
    import torch

    import paper_2607_05920_gb300 as fhe

    N, logQ = 1 << 12, 200
    ctx = fhe.Context(12, logQ, logQ)
    ctx.keygen(31)
    g = fs.rng(31)
    z1, z2 = fs.unit_disk(g, N // 2), fs.unit_disk(g, N // 2)
    enc = lambda z, seed: ctx.encrypt(fhe.fhe_ckks_encode(ctx, torch.from_numpy(z[None]).cuda(), 40, logQ), seed,  # noqa
                                      log_scale=40)
    out = ctx.mult_relin_rescale(enc(z1, 1), enc(z2, 2), 40)
    z = fhe.fhe_ckks_decode(ctx, ctx.decrypt(out), out.logQ, out.log_scale).cpu().numpy()[0]
    assert np.abs(z - z1 * z2).max() <= 2.0 ** -20
    ctx.close()


def _bgv_ctx(logN):
    import paper_2607_05920_gb300 as fhe

    t, levels = 65537, 8
    q0, r = bgv.chain_moduli(t, 54, 48)
    logQ = (q0 * r ** levels).bit_length()
    ctx = fhe.Context(logN, logQ, logQ, scheme=fhe.FHE_SCHEME_BGV, t=t, bgv_q0=q0, bgv_r=r, bgv_levels=levels)
    return fhe, ctx, t, logQ


def test_bgv_slots_match_oracle_and_multiply_slotwise():
    import torch

    fhe, ctx, t, logQ = _bgv_ctx(10)
    N = ctx.N
    g = fs.rng(620)
    x = fs.uniform_mod_t(g, (2,), N, t)
    y = fs.uniform_mod_t(g, (2,), N, t)
    pt = fhe.fhe_bgv_encode(ctx, to_dev(x.astype(np.int32)), logQ)
    host = pt.cpu().numpy().view(np.uint32)
    assert not host[:, 1:].any()
    for c in range(2):
        assert [int(v) for v in host[c, 0]] == bgv.slot_encode([int(v) for v in x[c]], N, t)
    # decode is the inverse, and equals the oracle's evaluation at the roots
    assert torch.equal(fhe.fhe_bgv_decode(ctx, pt[:, 0].contiguous()).cpu(), torch.from_numpy(x.astype(np.int32)))
    coeffs = fs.uniform_mod_t(g, (1,), N, t)
    got = fhe.fhe_bgv_decode(ctx, to_dev(coeffs.astype(np.int32))).cpu().numpy()[0]
    assert [int(v) for v in got] == bgv.slot_decode([int(v) for v in coeffs[0]], N, t)
    # slot-wise product through encryption, multiplication and decryption
    ctx.keygen(7)
    ca = ctx.encrypt(pt, 1)
    cb = ctx.encrypt(fhe.fhe_bgv_encode(ctx, to_dev(y.astype(np.int32)), logQ), 2)
    prod = fhe.fhe_bgv_decode(ctx, ctx.decrypt(ctx.mult_relin(ca, cb))).cpu().numpy()
    assert np.array_equal(prod.astype(np.int64), (x * y) % t)
    ctx.close()


def test_bgv_slots_workload_ring_roundtrip():
    import torch

    fhe, ctx, t, logQ = _bgv_ctx(14)
    x = fs.uniform_mod_t(fs.rng(621), (3,), ctx.N, t).astype(np.int32)
    pt = fhe.fhe_bgv_encode(ctx, to_dev(x), logQ)
    assert torch.equal(fhe.fhe_bgv_decode(ctx, pt[:, 0].contiguous()).cpu(), torch.from_numpy(x))
    ctx.close()
