"""The library's host sampler (fhe_sample, CPU only) against the oracle's sampler.

The library and the oracle implement Philox4x32-10 and the coefficient rules
separately; the oracle's is pinned by known answers and distribution checks
(tests/test_oracle_sampler.py).  Every word and coefficient must agree.
"""
import ctypes

import numpy as np
import pytest

from oracle import sampler as S


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEFCAFEF00D, (1 << 64) - 1])
def test_uniform_limbs_match(seed):
    import paper_2607_05920_gb300 as fhe

    for bits, tag1 in ((1200, 0), (97, 12345), (32, 7), (2400, 2 ** 32 - 1)):
        got = fhe.fhe_sample(seed, 4, tag1, fhe.FHE_SAMPLE_UNIFORM, 1000, bits)
        assert np.array_equal(got, S.uniform_limbs(seed, 4, tag1, 1000, bits)), bits


def test_ternary_hwt_gaussian_match():
    import paper_2607_05920_gb300 as fhe

    for seed in (3, 99, 1 << 40):
        assert np.array_equal(fhe.fhe_sample(seed, 1, 0, fhe.FHE_SAMPLE_TERNARY, 1 << 14),
                              S.ternary(seed, 1, 0, 1 << 14))
        for n, h in ((1 << 15, 64), (1 << 11, 2048), (8, 3)):
            assert np.array_equal(fhe.fhe_sample(seed, 1, 0, fhe.FHE_SAMPLE_HWT, n, h),
                                  S.sparse_ternary(seed, 1, 0, n, h)), (n, h)
        for sigma in (3.2, 1.0, 7.5):
            assert np.array_equal(fhe.fhe_sample(seed, 9, 5, fhe.FHE_SAMPLE_GAUSSIAN, 1 << 15, 0, sigma),
                                  S.gaussian(seed, 9, 5, 1 << 15, sigma)), sigma


def test_sample_rejects_bad_arguments():
    import paper_2607_05920_gb300 as fhe

    out = np.zeros(64, dtype=np.int32)
    for kind, n, param, sigma in ((7, 8, 0, 3.2), (fhe.FHE_SAMPLE_HWT, 8, 9, 3.2), (fhe.FHE_SAMPLE_GAUSSIAN, 8, 0, 0.0),
                                  (fhe.FHE_SAMPLE_GAUSSIAN, 8, 0, 11.0), (fhe.FHE_SAMPLE_UNIFORM, 8, 0, 3.2),
                                  (fhe.FHE_SAMPLE_TERNARY, 0, 0, 3.2)):
        assert fhe.lib.fhe_sample(1, 1, 0, kind, n, param, sigma, out.ctypes.data) == fhe.FHE_EINVAL


def test_ctx_create_rejects_bad_secret_and_error_parameters():
    import paper_2607_05920_gb300 as fhe

    h = ctypes.c_void_p()
    for hw, sigma in ((-1, 0.0), (2049, 0.0), (0, -1.0), (0, 10.5)):
        p = fhe.FheParams(0, 11, 100, 100, 0, 0, 0, 0, 0, hw, sigma)
        rc = fhe.lib.fhe_ctx_create(ctypes.byref(p), fhe.ALLOC_FN(), fhe.FREE_FN(), None, ctypes.byref(h))
        assert rc == fhe.FHE_EINVAL, (hw, sigma)
