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


@pytest.mark.parametrize("branches", [False, True])
def test_batched_graph_equals_per_op_and_oracle(branches):
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
    runner.capture(plan, branches=branches)
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


def test_form_search_gives_identical_results_at_the_batched_ring_sizes():
    """Rings 2^13 and 2^16 (two-pass transforms, tensor-core and integer forms): every kernel form of a group
    gives the same ciphertexts; the tuned graph equals per-level CipherTensor calls and per-op calls."""
    import torch

    from paper_2607_05920_gb300 import batch

    pairs = {13: make_pair(13, 1200, 1200, seed=54), 16: make_pair(16, 1200, 1200, seed=55)}
    ctxs = {k: p.ctx for k, p in pairs.items()}
    items = _items(pairs, 6, 56, 200, 1200)
    for logN in (13, 16):  # both rings present, one item near the top level
        N = 1 << logN
        from paper_2607_05920_gb300 import Ciphertext

        la = fs.uniform_limbs(fs.rng(logN), (1, 2), N, 1190)
        lb = fs.uniform_limbs(fs.rng(logN + 1), (1, 2), N, 1190)
        items.append(batch.Item(logN, 1190, Ciphertext(to_dev(la), 1190), Ciphertext(to_dev(lb), 1190)))
    runner = batch.BatchRunner(ctxs, 40)
    plan = runner.plan(items, {13: [1200], 16: [1200]})
    runner.pack(plan, items)
    outs = []
    for f in batch.FORMS:
        for g in plan.groups:
            runner.run_group(g, f)
        torch.cuda.synchronize()
        outs.append([g.O.clone() for g in plan.groups])
    for o in outs[1:]:
        assert all(torch.equal(x, y) for x, y in zip(o, outs[0]))
    tuner = batch.Autotuner()
    tuner.tune_forms(runner, plan, reps=1)
    assert all(g.forms in batch.FORMS for g in plan.groups)
    timings = tuner.tune_branches(runner, plan, reps=1)
    assert set(timings) == {"sequence", "branches"}
    runner.capture(plan)
    for g in plan.groups:
        g.O.zero_()
    runner.graph.replay()
    torch.cuda.synchronize()
    got = runner.outputs(plan, items)
    ref, lev = runner.per_op(items), runner.per_level(items)
    torch.cuda.synchronize()
    for i in range(len(items)):
        assert torch.equal(got[i], ref[i].data[0]) and torch.equal(got[i], lev[i]), i
    for p in pairs.values():
        p.ctx.close()
