"""Pins for the oracle's counter-based sampler (CPU only).

The generator is pinned to the published known-answer values of
Philox4x32-10; the coefficient rules are pinned to the distributions the
scheme asks for (Sec. 2 / Sec. 6: uniform ternary or Hamming-weight secrets,
rounded Gaussian errors with sigma = 3.2, uniform key parts).
"""
import os

import numpy as np

from oracle import sampler as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([[int(t, 16) for t in part.split()] for part in line.split("|")])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = S.philox4x32_10([np.uint64(c) for c in ctr], [np.uint64(k) for k in key])
        assert [int(x) for x in got] == want


def test_word_stream_layout():
    # word j is component j mod 4 of block j div 4, the block index in the counter's first word
    w = S.words(7, 3, 9, 12)
    for blk in range(3):
        out = S.philox4x32_10([np.uint64(blk), np.uint64(0), np.uint64(3), np.uint64(9)],
                              [np.uint64(7), np.uint64(0)])
        assert [int(x) for x in w[4 * blk:4 * blk + 4]] == [int(x) for x in out]
    # an offset start continues the same stream; the 64-bit seed splits into the key words
    assert np.array_equal(S.words(7, 3, 9, 5, start=7), w[7:12])
    hi = S.words((5 << 32) | 7, 3, 9, 4)
    out = S.philox4x32_10([np.uint64(0), np.uint64(0), np.uint64(3), np.uint64(9)], [np.uint64(7), np.uint64(5)])
    assert [int(x) for x in hi] == [int(x) for x in out]


def test_uniform_limbs_masks_the_top_limb_and_is_uniform():
    u = S.uniform_limbs(1, 2, 0, 1 << 14, 97)
    assert u.shape == (4, 1 << 14) and u.dtype == np.uint32
    assert int(u[3].max()) == 1  # 97 = 3 * 32 + 1 bits
    full = u[:3].astype(np.float64)
    assert abs(full.mean() / 2.0 ** 31 - 1.0) < 0.01
    # every bit of the full limbs is set about half the time
    bits = np.unpackbits(u[:3].view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005


def test_ternary_is_uniform_over_minus_one_zero_one():
    t = S.ternary(2, 1, 0, 1 << 16)
    counts = np.array([(t == v).sum() for v in (-1, 0, 1)])
    assert counts.sum() == 1 << 16
    # chi-square with 2 degrees of freedom well below its 0.999 quantile (13.8)
    exp = (1 << 16) / 3.0
    assert ((counts - exp) ** 2 / exp).sum() < 13.8
    # the rule itself on hand-picked words: floor(3 w / 2^32) - 1
    for w, v in ((0, -1), (0x55555555, -1), (0x55555556, 0), (0xAAAAAAAA, 0), (0xAAAAAAAB, 1), (0xFFFFFFFF, 1)):
        assert (w * 3) >> 32 == v + 1


def test_sparse_ternary_has_exactly_h_distinct_positions():
    for n, h in ((1 << 15, 64), (64, 64), (16, 5)):
        s = S.sparse_ternary(3, 1, 0, n, h)
        assert (s != 0).sum() == h and set(np.unique(s)) <= {-1, 0, 1}
    # positions spread over the whole ring and signs balanced, over many seeds
    pos = np.concatenate([np.nonzero(S.sparse_ternary(seed, 1, 0, 1024, 32))[0] for seed in range(200)])
    hist = np.bincount(pos // 128, minlength=8)
    exp = len(pos) / 8.0
    assert ((hist - exp) ** 2 / exp).sum() < 24.3  # chi-square, 7 dof, 0.999 quantile
    signs = np.concatenate([S.sparse_ternary(seed, 1, 0, 1024, 32) for seed in range(200)])
    assert abs(int(signs.sum())) < 4 * np.sqrt(200 * 32)


def test_gaussian_table_and_samples():
    B, thr = S.gaussian_thresholds(3.2)
    assert B == 19 and len(thr) == 38
    assert all(a <= b for a, b in zip(thr, thr[1:])) and thr[-1] < 1 << 32
    # symmetric: P(e <= -k - 1) = P(e >= k + 1), within the 2^-32 rounding of each threshold
    for k in range(19):
        lower = thr[19 - k - 1]             # P(e <= -k-1) 2^32
        upper = (1 << 32) - thr[19 + k]     # P(e >= k+1) 2^32
        assert abs(lower - upper) <= 2
    # P(0) = rho(0) / sum rho = 1 / sum_k exp(-k^2 / 20.48)
    p0 = 1.0 / sum(np.exp(-k * k / 20.48) for k in range(-19, 20))
    assert abs((thr[19] - thr[18]) / 2.0 ** 32 - p0) < 1e-9
    e = S.gaussian(4, 3, 0, 1 << 18)
    assert e.dtype == np.int32 and int(np.abs(e).max()) <= 19
    assert abs(e.mean()) < 0.05 and abs(e.std() - 3.2) < 0.03
    # the rule on words at and around the thresholds
    t = np.array(thr, dtype=np.int64)
    for i in (0, 18, 19, 37):
        for w, want in ((thr[i] - 1, i - 19), (thr[i], i - 18)):
            assert int(np.searchsorted(t, w, side="right")) - 19 == want
