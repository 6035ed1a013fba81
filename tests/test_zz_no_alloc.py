"""fhe_mult_relin_rescale_noalloc against fhe_mult_relin_rescale (needs a GB300).

The no-allocation entry point serves callers that cannot allocate device
memory where they multiply (hosts that forbid allocation after start-up,
plug-ins that must not touch the device allocator).  It must give the same
ciphertexts, bit for bit, as the workspace entry point, call after call,
even though every call reuses one static scratch array.  This file is named
so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import fhe_synth as fs

pytestmark = pytest.mark.gpu


def _pair_setup():
    import torch

    import paper_2607_05920_gb300 as fhe

    logN, logQ, logP = 11, 120, 120
    N = 1 << logN
    g = fs.rng(4242)
    ctx = fhe.Context(logN, logQ, logP)
    ctx.keygen_inject(fs.ternary(g, (), N), fs.uniform_limbs(g, (), N, logQ), fs.gaussian(g, (), N),
               fs.uniform_limbs(g, (), N, logQ + logP), fs.gaussian(g, (), N))

    def rand_ct(cnum):
        a = fs.uniform_limbs(g, (cnum, 2), N, logQ).view(np.int32)
        return fhe.Ciphertext(torch.from_numpy(a.copy()).cuda(), logQ)

    return fhe, ctx, rand_ct


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    import torch

    fhe, ctx, rand_ct = _pair_setup()
    k = 30
    for call in range(2):  # two calls in a row: the static scratch keeps the previous call's contents
        a, b = rand_ct(3), rand_ct(3)
        want = ctx.empty_ct(3, a.logQ - k)
        fhe.fhe_mult_relin_rescale(ctx, a, b, k, want)
        got = ctx.empty_ct(3, a.logQ - k)
        ca, cb, co = a.c(), b.c(), got.c()
        rc = fhe.lib.fhe_mult_relin_rescale_noalloc(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), k,
                                                    ctypes.byref(co),
                                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == fhe.FHE_OK, fhe.lib.fhe_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got.data, want.data), f"call {call}: differs from fhe_mult_relin_rescale"
    ctx.close()


def test_noalloc_rejects_work_beyond_the_static_scratch():
    import torch

    fhe, ctx, rand_ct = _pair_setup()
    # 64 pairs at N = 2^11, logQ = 120 need more than 32 MiB of scratch
    assert fhe.lib.fhe_workspace_bytes(ctx.handle, fhe.FHE_OP_MULT, 120, 64) > (32 << 20)
    a, b = rand_ct(64), rand_ct(64)
    out = ctx.empty_ct(64, 90)
    ca, cb, co = a.c(), b.c(), out.c()
    rc = fhe.lib.fhe_mult_relin_rescale_noalloc(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), 30, ctypes.byref(co),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == fhe.FHE_EINVAL
    assert b"static scratch" in fhe.lib.fhe_last_error()
    # argument errors come first, as for fhe_mult_relin_rescale: k < 1 is rejected whatever the size
    rc = fhe.lib.fhe_mult_relin_rescale_noalloc(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), 0, ctypes.byref(co),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == fhe.FHE_EINVAL
    assert b"k >= 1" in fhe.lib.fhe_last_error()
    ctx.close()
