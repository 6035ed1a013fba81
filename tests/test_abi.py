"""The C-ABI library loads, exports every entry point include/fhe.h declares,
and its host-only helpers answer without a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fhe.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fhe_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_scheme_calls():
    names = _declared()
    for must in ("fhe_keygen", "fhe_encrypt", "fhe_mult_relin", "fhe_rescale", "fhe_rotate", "fhe_decrypt"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2607_05920_gb300 as fhe

    lib = ctypes.CDLL(fhe.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared calls
    assert sorted(fhe.SIGNATURES) == _declared()


def test_host_helpers_without_gpu():
    import paper_2607_05920_gb300 as fhe

    assert fhe.lib.fhe_ct_bytes(16, 1200, 1) == 2 * 38 * 65536 * 4
    assert fhe.lib.fhe_ct_bytes(11, 120, 3) == 3 * 2 * 4 * 2048 * 4
    assert fhe.lib.fhe_ct_bytes(17, 120, 1) == 0
    # prime counts: prod of all but the top prime covers 2^bound (primes in (2^29, 2^30))
    for bits in (1, 30, 31, 100, 1217, 2417, 3616):
        r = fhe.fhe_primes_for_bound(bits)
        assert r >= 2
        assert 30 * (r - 1) >= bits
        assert 29 * (r - 2) < bits
    assert fhe.fhe_primes_for_bound(3616) == 123  # relinearisation at N=2^16, logQ=logP=1200
    assert fhe.fhe_primes_for_bound(2417) == 82   # Karatsuba tensor product, same ring


def test_ctx_create_rejects_bad_params_before_touching_the_device():
    import paper_2607_05920_gb300 as fhe

    h = ctypes.c_void_p()
    for prm in ((0, 2, 100, 100, 0), (0, 17, 100, 100, 0), (1, 11, 100, 100, 0), (0, 11, 0, 100, 0),
                (0, 11, 3000, 3000, 0), (0, 11, 100, 100, 4), (0, 11, 100, 100, -1)):
        p = fhe.FheParams(*prm)
        rc = fhe.lib.fhe_ctx_create(ctypes.byref(p), fhe.ALLOC_FN(), fhe.FREE_FN(), None, ctypes.byref(h))
        assert rc == fhe.FHE_EINVAL
        assert fhe.lib.fhe_last_error()
    rc = fhe.lib.fhe_ctx_create(None, fhe.ALLOC_FN(), fhe.FREE_FN(), None, ctypes.byref(h))
    assert rc == fhe.FHE_EINVAL


def test_product_path_does_not_import_the_oracle():
    # the package and the bench's GPU leg must not reach into oracle/
    pkg = os.path.join(ROOT, "paper_2607_05920_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_batch_call_rejects_empty_or_oversized_group_lists_before_touching_the_device():
    import paper_2607_05920_gb300 as fhe

    assert fhe.lib.fhe_mult_relin_rescale_batch(None, 1, 40, None, None) == fhe.FHE_EINVAL
    arr = (fhe.FheBatchGroup * 33)()
    for n in (0, 33):
        assert fhe.lib.fhe_mult_relin_rescale_batch(arr, n, 40, None, None) == fhe.FHE_EINVAL
    assert fhe.lib.fhe_mult_relin_rescale_batch(arr, 1, -1, None, None) == fhe.FHE_EINVAL
    assert b"batch" in fhe.lib.fhe_last_error()
