"""Uneven batches (several ring sizes and levels) run as one CUDA graph (needs a GB300).

Every ciphertext of the batched form must equal the per-op result of the same
pair, bit for bit, and a sample must equal the oracle's multiplication at the
pair's own level.
"""
import numpy as np
import pytest

import fhe_synth as fs
from oracle import bigint, ckks

from fhe_setup import make_pair, to_dev

pytestmark = pytest.mark.gpu


def _items(pairs, count, seed, lo, hi):
    import paper_2607_05920_gb300 as fhe
    from paper_2607_05920_gb300 import batch

    g = fs.rng(seed)
    items = []
    rings = sorted(pairs)
    for _ in range(count):
        logN = rings[int(g.integers(0, len(rings)))]
        logQ = int(g.integers(lo, hi + 1))
        N = 1 << logN
        la = fs.uniform_limbs(g, (1, 2), N, logQ)
        lb = fs.uniform_limbs(g, (1, 2), N, logQ)
        items.append(batch.Item(logN, logQ, fhe.Ciphertext(to_dev(la), logQ), fhe.Ciphertext(to_dev(lb), logQ)))
    return items


def test_batched_graph_equals_per_op_and_oracle():
    import torch

    from paper_2607_05920_gb300 import batch

    pairs = {11: make_pair(11, 300, 300, seed=51), 12: make_pair(12, 300, 300, seed=52)}
    ctxs = {k: p.ctx for k, p in pairs.items()}
    k = 30
    items = _items(pairs, 24, 53, 100, 300)
    runner = batch.BatchRunner(ctxs, k)
    tuned = batch.Autotuner().tune(runner, items, reps=1)
    sched = tuned["schedule"]
    for logN, bounds in sched.items():
        assert bounds == sorted(bounds) and bounds[-1] >= max(it.logQ for it in items if it.logN == logN)
    plan = runner.plan(items, sched)
    runner.pack(plan, items)
    runner.capture(plan)
    for g in plan.groups:
        g.O.zero_()
    runner.graph.replay()
    torch.cuda.synchronize()
    got = runner.outputs(plan, items)
    ref = runner.per_op(items)
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        assert torch.equal(got[i], ref[i].data[0]), (i, it.logN, it.logQ)
    # sample against the oracle at the pair's own level
    for i in (0, 5, 17):
        it = items[i]
        P = pairs[it.logN]
        oa = tuple(bigint.from_limbs(it.a.data.cpu().numpy().view(np.uint32)[0, p]) for p in range(2))
        ob = tuple(bigint.from_limbs(it.b.data.cpu().numpy().view(np.uint32)[0, p]) for p in range(2))
        want = ckks.rescale(ckks.mult(oa, ob, P.evk, it.logQ, 300), k, it.logQ)
        host = got[i].cpu().numpy().view(np.uint32)
        assert tuple(bigint.from_limbs(host[p]) for p in range(2)) == tuple(want)
    for p in pairs.values():
        p.ctx.close()


def test_bucket_bounds_cover_and_split():
    from paper_2607_05920_gb300 import batch

    lv = [200, 250, 300, 700, 710, 1200, 1199, 640]
    for nb in (1, 2, 3, 4, 8, 20):
        b = batch.bucket_bounds(lv, nb)
        assert b[-1] == 1200 and b == sorted(set(b)) and len(b) <= min(nb, len(lv))
    assert batch.bucket_bounds(lv, 1) == [1200]
