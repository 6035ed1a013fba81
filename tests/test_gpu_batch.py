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
    # the work-table call at these widths (82 / 123 primes at the top level): the same ciphertexts
    for sc in ((0, 0, 1), (3, 4, 4)):
        for g in plan.groups:
            g.O.zero_()
        runner.run_table(plan, sc)
        torch.cuda.synchronize()
        got = runner.outputs(plan, items)
        assert all(torch.equal(got[i], ref[i].data[0]) for i in range(len(items))), sc
    for p in pairs.values():
        p.ctx.close()


def test_work_table_call_equals_per_op_at_every_schedule():
    """Five ring sizes (2^12 runs per group inside the call, 2^13..2^16 through the work-table launches, all four
    column-pass shapes), two level buckets on one ring: every schedule of the work-table call, eager and
    graph-captured, gives the per-op ciphertexts bit for bit; two items match the oracle at their own level."""
    import torch

    from paper_2607_05920_gb300 import batch

    rings = (12, 13, 14, 15, 16)
    pairs = {n: make_pair(n, 500, 500, seed=60 + n) for n in rings}
    ctxs = {n: p.ctx for n, p in pairs.items()}
    k = 40
    items = _items(pairs, 8, 57, 100, 500)
    for n in rings:  # every ring present, one item near the top level
        items += _items({n: None}, 1, 70 + n, 450, 500)
    runner = batch.BatchRunner(ctxs, k)
    sched = {n: [500] for n in rings}
    sched[14] = [300, 500]
    plan = runner.plan(items, sched)
    runner.pack(plan, items)
    ref = runner.per_op(items)
    torch.cuda.synchronize()
    for sc, per_ring in (((0, 0, 1), False), ((3, 4, 4), False), ((2, 2, 16), False), ((1, 1, 3), False),
                         (None, False), ((0, 0, 1), True)):
        for g in plan.groups:
            g.O.zero_()
        runner.run_table(plan, sc, per_ring)
        torch.cuda.synchronize()
        got = runner.outputs(plan, items)
        for i, it in enumerate(items):
            assert torch.equal(got[i], ref[i].data[0]), (sc, per_ring, i, it.logN, it.logQ)
    runner.table, runner.table_per_ring = (2, 4, 4), True  # one call per ring, rings as graph branches
    runner.capture(plan)
    for _ in range(2):
        for g in plan.groups:
            g.O.zero_()
        runner.graph.replay()
        torch.cuda.synchronize()
        got = runner.outputs(plan, items)
        assert all(torch.equal(got[i], ref[i].data[0]) for i in range(len(items)))
    for i in (next(j for j, it in enumerate(items) if it.logN == 13),
              next(j for j, it in enumerate(items) if it.logN == 15)):
        it = items[i]
        P = pairs[it.logN]
        oa = tuple(bigint.from_limbs(it.a.data.cpu().numpy().view(np.uint32)[0, p]) for p in range(2))
        ob = tuple(bigint.from_limbs(it.b.data.cpu().numpy().view(np.uint32)[0, p]) for p in range(2))
        want = ckks.rescale(ckks.mult(oa, ob, P.evk, it.logQ, 500), k, it.logQ)
        host = got[i].cpu().numpy().view(np.uint32)
        assert tuple(bigint.from_limbs(host[p]) for p in range(2)) == tuple(want)
    for p in pairs.values():
        p.ctx.close()


def test_work_table_call_rejects_bad_groups():
    import torch

    import paper_2607_05920_gb300 as fhe
    from paper_2607_05920_gb300 import batch

    p = make_pair(13, 300, 300, seed=80)
    items = _items({13: None}, 2, 81, 100, 300)
    runner = batch.BatchRunner({13: p.ctx}, 30)
    plan = runner.plan(items, {13: [150, 300]})
    if len(plan.groups) < 2:
        plan = runner.plan(items, {13: [300]})
    g = plan.groups[0]
    ws = runner.group_ws(g)
    base = (p.ctx, g.A, g.B, g.O, g.bits, g.logQ_max)
    with pytest.raises(fhe.FheError):  # two groups on one workspace
        fhe.fhe_mult_relin_rescale_batch([base + (ws,), base + (ws,)], 30)
    with pytest.raises(fhe.FheError):  # out aliases a
        fhe.fhe_mult_relin_rescale_batch([(p.ctx, g.A, g.B, g.A, g.bits, g.logQ_max, ws)], 30)
    with pytest.raises(fhe.FheError):  # workspace too small
        fhe.fhe_mult_relin_rescale_batch([base + (ws[:1024],)], 30)
    with pytest.raises(fhe.FheError):  # bad schedule
        fhe.fhe_mult_relin_rescale_batch([base + (ws,)], 30, (1, 1, 0))
    torch.cuda.synchronize()
    p.ctx.close()
