"""The continuous-batching server (needs a GB300).

Each request's ciphertext must be identical whether it was served in a mix of
concurrent requests (batched across levels, overlapping streams) or alone;
a sampled multiplication must also equal the oracle's.
"""
import copy

import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, ckks

from fhe_setup import make_pair, to_dev

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_results_and_oracle():
    import torch

    import paper_2607_05920_gb300 as fhe
    from paper_2607_05920_gb300 import serve

    steps = [1, 2, 4]
    P = make_pair(12, 600, 600, seed=61, rot_steps=steps)
    ctx = P.ctx
    g = fs.rng(62)
    levels = [600, 560, 520]
    pool = {lq: fhe.Ciphertext(to_dev(fs.uniform_limbs(g, (4, 2), ctx.N, lq)), lq) for lq in levels}
    reqs = serve.make_requests(g, rate_hz=600.0, duration_s=0.08, levels=levels, pool_size=4, steps=steps)
    assert len(reqs) >= 20 and {r.op for r in reqs} == {"mult", "rotate", "poly7"}
    srv = serve.Server(ctx, pool, k=40, budget_bytes=2 << 30, max_batch=16, streams=2)
    served = copy.deepcopy(reqs)
    stats = srv.run(served)
    torch.cuda.synchronize()
    assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    by_id = {r.rid: r for r in served}
    picks = [r for r in reqs if r.op == "mult"][:2] + [r for r in reqs if r.op == "rotate"][:2] + \
        [r for r in reqs if r.op == "poly7"][:2]
    for r in picks:
        alone = copy.deepcopy(r)
        alone.t_arrive = 0.0
        srv1 = serve.Server(ctx, pool, k=40, budget_bytes=2 << 30, max_batch=16, streams=1)
        srv1.run([alone])
        torch.cuda.synchronize()
        assert torch.equal(alone.result, by_id[r.rid].result), (r.rid, r.op, r.logQ)
    # one multiplication against the oracle at its own level
    r = [r for r in reqs if r.op == "mult"][0]
    ha = pool[r.logQ].data.cpu().numpy().view(np.uint32)
    oa = tuple(bigint.from_limbs(ha[r.a, p]) for p in range(2))
    ob = tuple(bigint.from_limbs(ha[r.b, p]) for p in range(2))
    want = ckks.rescale(ckks.mult(oa, ob, P.evk, r.logQ, 600), 40, r.logQ)
    host = by_id[r.rid].result.cpu().numpy().view(np.uint32)
    assert tuple(bigint.from_limbs(host[p]) for p in range(2)) == tuple(want)
    ctx.close()


def test_injected_failures_fail_only_their_own_requests():
    """A completion callback that raises and a batch whose stream reports an error (both injected on the
    host): the server completes every other request, with the same results as the plain per-op path."""
    import torch

    import paper_2607_05920_gb300 as fhe
    from paper_2607_05920_gb300 import serve

    steps = [1, 2]
    P = make_pair(12, 400, 400, seed=63, rot_steps=steps)
    ctx = P.ctx
    g = fs.rng(64)
    levels = [400, 360]
    pool = {lq: fhe.Ciphertext(to_dev(fs.uniform_limbs(g, (3, 2), ctx.N, lq)), lq) for lq in levels}
    reqs = serve.make_requests(g, rate_hz=500.0, duration_s=0.06, levels=levels, pool_size=3, steps=steps)
    assert len(reqs) >= 15
    calls = {"n": 0}
    bad_cb = {r.rid for r in reqs[::5]}

    def on_done(r):
        calls["n"] += 1
        if r.rid in bad_cb:
            raise RuntimeError("callback failed")

    batches = {"n": 0}

    def fail_batch(si, tasks):  # the second batch that completes reports a stream error
        batches["n"] += 1
        return batches["n"] == 2

    srv = serve.Server(ctx, pool, k=40, budget_bytes=2 << 30, max_batch=8, streams=2, fail_batch=fail_batch)
    served = copy.deepcopy(reqs)
    stats = srv.run(served, on_done=on_done)
    torch.cuda.synchronize()
    failed = [r for r in served if r.error.startswith("stream")]
    assert stats["failed"] == len(failed) >= 1
    assert stats["completed"] + stats["failed"] == len(reqs)
    assert stats["callback_errors"] == sum(1 for r in served if r.error.startswith("callback"))
    assert calls["n"] == stats["completed"]
    alone = copy.deepcopy(reqs)
    serve.run_per_op(ctx, pool, alone, 40)
    by_id = {r.rid: r for r in alone}
    for r in served:
        if not r.error.startswith("stream"):
            assert torch.equal(r.result, by_id[r.rid].result), (r.rid, r.op)
    ctx.close()


def test_served_mult_at_the_serving_modulus_matches_oracle():
    """logQ = logP = 1550 (the serving workload's top level) on a ring of 2^12: served multiplications at two
    levels, ragged in one batch, equal the oracle's."""
    import paper_2607_05920_gb300 as fhe
    from paper_2607_05920_gb300 import serve

    P = make_pair(12, 1550, 1550, seed=65)
    ctx = P.ctx
    g = fs.rng(66)
    levels = [1550, 1540]  # both 49 limbs: one ragged batch
    pool = {lq: fhe.Ciphertext(to_dev(fs.uniform_limbs(g, (2, 2), ctx.N, lq)), lq) for lq in levels}
    reqs = [serve.Request(i, 0.0, "mult", levels[i % 2], i % 2, (i + 1) % 2) for i in range(4)]
    srv = serve.Server(ctx, pool, k=40, budget_bytes=4 << 30, max_batch=8, streams=2)
    stats = srv.run(reqs)
    assert stats["completed"] == 4
    for r in reqs[:2]:
        ha = pool[r.logQ].data.cpu().numpy().view(np.uint32)
        oa = tuple(bigint.from_limbs(ha[r.a, p]) for p in range(2))
        ob = tuple(bigint.from_limbs(ha[r.b, p]) for p in range(2))
        want = ckks.rescale(ckks.mult(oa, ob, P.evk, r.logQ, 1550), 40, r.logQ)
        host = r.result.cpu().numpy().view(np.uint32)
        assert tuple(bigint.from_limbs(host[p]) for p in range(2)) == tuple(want), r.logQ
    ctx.close()
