"""Failure detection on the GPU without faulting it (needs a GB300).

Every device-side wait of the library's pipelined kernels is bounded: when it
runs out it sets a status word and returns, and fhe_sync reports
FHE_ETIMEOUT.  The self-test kernel waits on a barrier that nothing arms, with
a limit of a few hundred polls, so the wait runs out within milliseconds.  The
context must stay usable afterwards.
"""
import numpy as np
import pytest

from oracle import ckks

from fhe_setup import ct_ints, make_pair, random_ct_limbs, to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_is_reported():
    import torch

    import paper_2607_05920_gb300 as fhe

    P = make_pair(11, 120, 120, seed=501)
    stream = torch.cuda.current_stream().cuda_stream
    assert fhe.lib.fhe_sync(P.ctx.handle) == fhe.FHE_OK
    assert fhe.lib.fhe_selftest_wait_timeout(200, stream) == fhe.FHE_OK
    assert fhe.lib.fhe_sync(P.ctx.handle) == fhe.FHE_ETIMEOUT
    assert b"bounded device-side wait" in fhe.lib.fhe_last_error()
    # reported once, then cleared
    assert fhe.lib.fhe_sync(P.ctx.handle) == fhe.FHE_OK
    # the context still works: a multiplication after the timeout matches the oracle
    la = random_ct_limbs(P.g, 1, 2048, 120)
    lb = random_ct_limbs(P.g, 1, 2048, 120)
    out = P.ctx.mult_relin_rescale(fhe.Ciphertext(to_dev(la), 120), fhe.Ciphertext(to_dev(lb), 120), 30)
    from oracle import bigint

    oa = tuple(bigint.from_limbs(la[0, p]) for p in range(2))
    ob = tuple(bigint.from_limbs(lb[0, p]) for p in range(2))
    assert ct_ints(out)[0] == tuple(ckks.rescale(ckks.mult(oa, ob, P.evk, 120, 120), 30, 120))
    assert fhe.lib.fhe_sync(P.ctx.handle) == fhe.FHE_OK
    assert fhe.lib.fhe_selftest_wait_timeout(0, stream) == fhe.FHE_EINVAL
    P.ctx.close()
