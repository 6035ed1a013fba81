"""Shared set-up for the GPU parity tests: the same seeded keys and noise on both sides.

The random polynomials come from fhe_synth; the CUDA library receives them
through its C ABI (fhe_keygen_inject / fhe_encrypt_inject), the oracle receives them as
Python integers.  Nothing here computes any part of the scheme.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import fhe_synth as fs
from oracle import bigint, ckks


@dataclass
class Pair:
    ctx: object          # paper_2607_05920_gb300.Context
    prm: ckks.CkksParams
    s: list
    pk: tuple
    evk: tuple
    g: np.random.Generator
    rtk: dict
    ck: tuple = None


def make_pair(logN, logQ, logP, seed, hwt=None, rot_steps=(), crt=0, conj=False):
    import paper_2607_05920_gb300 as fhe

    g = fs.rng(seed)
    N = 1 << logN
    s = fs.sparse_ternary(g, N, hwt) if hwt else fs.ternary(g, (), N)
    a_pk = fs.uniform_limbs(g, (), N, logQ)
    e_pk = fs.gaussian(g, (), N)
    a_ev = fs.uniform_limbs(g, (), N, logQ + logP)
    e_ev = fs.gaussian(g, (), N)
    ctx = fhe.Context(logN, logQ, logP, crt=crt)
    ctx.keygen_inject(s, a_pk, e_pk, a_ev, e_ev)
    prm = ckks.CkksParams(logN, logQ, logP)
    si = [int(x) for x in s]
    pk = ckks.public_key(prm, si, bigint.from_limbs(a_pk), [int(x) for x in e_pk])
    evk = ckks.relin_key(prm, si, bigint.from_limbs(a_ev), [int(x) for x in e_ev])
    rtk = {}
    for step in rot_steps:
        a = fs.uniform_limbs(g, (), N, logQ + logP)
        e = fs.gaussian(g, (), N)
        ctx.keygen_rotation(step, a, e)
        rtk[step] = ckks.rotation_key(prm, si, step, bigint.from_limbs(a), [int(x) for x in e])
    ck = None
    if conj:
        a = fs.uniform_limbs(g, (), N, logQ + logP)
        e = fs.gaussian(g, (), N)
        ctx.keygen_conjugation(a, e)
        ck = ckks.conjugation_key(prm, si, bigint.from_limbs(a), [int(x) for x in e])
    return Pair(ctx, prm, si, pk, evk, g, rtk, ck)


def to_dev(arr):
    import torch

    a = np.ascontiguousarray(arr)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a.copy()).cuda()


def encrypt_both(P: Pair, msgs, logQ=None):
    """Encrypt integer plaintext polynomials (list of lists) on both sides with shared noise."""
    import paper_2607_05920_gb300 as fhe

    N = P.prm.N
    lq = P.prm.logQ if logQ is None else logQ
    cnum = len(msgs)
    v = fs.ternary(P.g, (cnum,), N)
    e0 = fs.gaussian(P.g, (cnum,), N)
    e1 = fs.gaussian(P.g, (cnum,), N)
    mask = (1 << lq) - 1
    pt = np.stack([bigint.to_limbs([x & mask for x in m], fhe.limbs(lq)) for m in msgs])
    ct = P.ctx.encrypt_inject(to_dev(pt), to_dev(v), to_dev(e0), to_dev(e1), logQ=lq)
    octs = [ckks.encrypt(P.prm, P.pk, m, [int(x) for x in v[i]], [int(x) for x in e0[i]],
                         [int(x) for x in e1[i]], logQ=lq) for i, m in enumerate(msgs)]
    return ct, octs


def ct_ints(ct):
    """GPU ciphertext batch -> list over cnum of (b, a) lists of Python ints."""
    host = ct.data.cpu().numpy().view(np.uint32)
    return [tuple(bigint.from_limbs(host[c, p]) for p in range(2)) for c in range(host.shape[0])]


def random_ct_limbs(g, cnum, N, logQ):
    """Uniform ciphertexts (both polynomials uniform mod 2^logQ) as limbs (cnum, 2, L, N)."""
    return fs.uniform_limbs(g, (cnum, 2), N, logQ)
