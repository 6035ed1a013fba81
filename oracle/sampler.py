"""The counter-based sampler behind seeded key generation and encryption (test infrastructure).

The paper draws its secrets, errors, ephemeral polynomials and uniform key
parts (Sec. 2 "Fully Homomorphic Encryption"; Sec. 6 "Cryptographic Key
Management": secret key, public key, relinearisation and rotation keys) but
names no generator.  Where a test cannot pass the random values in, the
library and this oracle each implement the same published counter-based
generator, Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random
Numbers: As Easy as 1, 2, 3", SC 2011), and the same rules that turn its
32-bit words into coefficients.  This module is the oracle's own
implementation, written from that definition; it shares no code with the
library.

Philox4x32-10 maps a 128-bit counter (c0, c1, c2, c3) and a 64-bit key
(k0, k1) to four 32-bit words by ten rounds of
    (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2            (full 64-bit products)
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key advanced by the Weyl
constants (0x9E3779B9, 0xBB67AE85) between rounds.

Word stream: word j of stream (seed, tag0, tag1) is component j mod 4 of
Philox(counter = (j div 4 mod 2^32, j div 2^34, tag0, tag1),
key = (seed mod 2^32, seed div 2^32)).

Coefficient rules (readings: the paper fixes only the distributions):
  uniform mod 2^bits  limb l of coefficient n is word l N + n, the top limb
                      masked to the bits above 32 (L - 1);
  ternary             word n -> floor(3 w / 2^32) - 1 in {-1, 0, 1};
  sparse ternary (h)  a partial Fisher-Yates shuffle of 0..N-1: for i < h,
                      swap positions i and i + floor((N - i) w_i / 2^32); the
                      coefficient at the i-th chosen position is +1 if bit 0
                      of w_(h+i) is 0 and -1 otherwise;
  rounded Gaussian    sigma (3.2), support |e| <= B = floor(6 sigma): weights
                      rho(k) = exp(-k^2 / (2 sigma^2)) for |k| <= B, running
                      sums S_k = S_(k-1) + rho(k) from k = -B in double
                      precision, thresholds T_k = floor(2^32 S_k / S_B) for
                      k = -B .. B-1; word n gives the smallest k with
                      w < T_k, or B.
Tags (tag0): 1 secret, 2 public-key a, 3 public-key e, 4 relinearisation-key
a, 5 its e, 6 / 7 switching key a / e of Galois element tag1 (rotations,
conjugation), 8 / 9 / 10 encryption v / e0 / e1 of ciphertext tag1.

Parity: pinned by the published known-answer values of Philox4x32-10 and by
distribution checks (tests/test_oracle_sampler.py).
"""
from __future__ import annotations

import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = 0xFFFFFFFF

TAG_SECRET, TAG_PK_A, TAG_PK_E, TAG_EV_A, TAG_EV_E, TAG_SW_A, TAG_SW_E = 1, 2, 3, 4, 5, 6, 7
TAG_ENC_V, TAG_ENC_E0, TAG_ENC_E1 = 8, 9, 10


def philox4x32_10(ctr, key):
    """One block: ctr (c0, c1, c2, c3), key (k0, k1), each component an array of 32-bit values."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) for k in key)
    for rnd in range(10):
        p0 = c0 * np.uint64(M0)
        p1 = c2 * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if rnd < 9:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK32)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK32)
    return c0, c1, c2, c3


def words(seed: int, tag0: int, tag1: int, count: int, start: int = 0) -> np.ndarray:
    """Words start .. start + count - 1 of stream (seed, tag0, tag1), uint32."""
    if count <= 0:
        return np.zeros(0, dtype=np.uint32)
    j = np.arange(start, start + count, dtype=np.uint64)
    blk = j >> np.uint64(2)
    ctr = (blk & np.uint64(MASK32), blk >> np.uint64(32), np.full_like(blk, tag0 & MASK32),
           np.full_like(blk, tag1 & MASK32))
    key = (np.uint64(seed & MASK32), np.uint64((seed >> 32) & MASK32))
    out = philox4x32_10(ctr, key)
    comp = (j & np.uint64(3)).astype(np.int64)
    stacked = np.stack(out)  # (4, count)
    return stacked[comp, np.arange(count)].astype(np.uint32)


def uniform_limbs(seed: int, tag0: int, tag1: int, n: int, bits: int) -> np.ndarray:
    """Uniform integers mod 2^bits as limbs (L, n), L = ceil(bits / 32)."""
    L = (bits + 31) // 32
    w = words(seed, tag0, tag1, L * n).reshape(L, n)
    top = bits - 32 * (L - 1)
    if top < 32:
        w[L - 1] &= np.uint32((1 << top) - 1)
    return w


def ternary(seed: int, tag0: int, tag1: int, n: int) -> np.ndarray:
    w = words(seed, tag0, tag1, n).astype(np.uint64)
    return ((w * np.uint64(3)) >> np.uint64(32)).astype(np.int64).astype(np.int8) - np.int8(1)


def sparse_ternary(seed: int, tag0: int, tag1: int, n: int, h: int) -> np.ndarray:
    w = [int(x) for x in words(seed, tag0, tag1, 2 * h)]
    perm = list(range(n))
    out = np.zeros(n, dtype=np.int8)
    for i in range(h):
        r = i + (((n - i) * w[i]) >> 32)
        perm[i], perm[r] = perm[r], perm[i]
        out[perm[i]] = -1 if (w[h + i] & 1) else 1
    return out


def gaussian_thresholds(sigma: float = 3.2) -> tuple[int, list[int]]:
    """(B, [T_-B, ..., T_(B-1)]) of the rounded-Gaussian rule above."""
    B = int(math.floor(6.0 * sigma))
    rho = [math.exp(-(k * k) / (2.0 * sigma * sigma)) for k in range(-B, B + 1)]
    # running sums in plain double addition, in order from k = -B (the total is the last one)
    run, acc = [], 0.0
    for x in rho:
        acc += x
        run.append(acc)
    total = run[-1]
    return B, [int(math.floor(run[i] / total * 4294967296.0)) for i in range(2 * B)]


def gaussian(seed: int, tag0: int, tag1: int, n: int, sigma: float = 3.2) -> np.ndarray:
    B, thr = gaussian_thresholds(sigma)
    w = words(seed, tag0, tag1, n).astype(np.int64)
    t = np.asarray(thr, dtype=np.int64)
    # number of thresholds <= w is the index of the first threshold above w
    return (np.searchsorted(t, w, side="right") - B).astype(np.int32)
