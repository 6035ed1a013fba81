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

