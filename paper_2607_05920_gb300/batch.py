"""Batched execution of many HMult+relin+rescale pairs at uneven ring sizes and levels.

The CipherTensor batch of the paper (Sec. 6, `cnum`) has one ring size and one
level.  A workload that mixes ring sizes (N = 2^13 .. 2^16) and levels is run
here as a plan of *groups*: one group per (ring, level bucket), each a single
`fhe_mult_relin_rescale_ragged` call over ciphertexts padded to the bucket's
widest level, with every ciphertext keeping its own modulus.  The plan's
launches (about 16 kernels per group) are captured once into a CUDA graph, so
the whole batch is one graph launch from the host.

The level buckets are the prime-count schedule: a wider bucket pads more
ciphertexts to more NTT primes and limbs, a narrower one costs more launches.
`Autotuner` measures candidate schedules on the batch at hand and keeps the
fastest per (GPU, ring size, batch size class).

All arithmetic runs in the library's kernels; this module only plans, packs
(device-to-device copies into padded tensors) and launches.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

from . import (FHE_OP_MULT, Ciphertext, Context, fhe_mult_relin_rescale, fhe_mult_relin_rescale_ragged, limbs)


@dataclass
class Item:
    """One ciphertext pair: both operands at modulus 2^logQ on ring 2^logN."""

    logN: int
    logQ: int
    a: Ciphertext
    b: Ciphertext


@dataclass
class Group:
    ctx: Context
    logN: int
    idx: list          # item indices
    logQ_max: int
    L_pad: int
    A: object = None   # (cnum, 2, L_pad, N) padded inputs / output
    B: object = None
    O: object = None
    bits: object = None


def bucket_bounds(levels: list[int], nbuckets: int) -> list[int]:
    """Upper bounds (inclusive, multiples of 32 bits where possible) splitting sorted levels into ~equal groups."""
    lv = sorted(levels)
    if not lv:
        return []
    nb = max(1, min(nbuckets, len(lv)))
    bounds = []
    for j in range(1, nb + 1):
        q = lv[min(len(lv) - 1, (j * len(lv)) // nb - 1)]
        bounds.append(q)
    return sorted(set(bounds))


@dataclass
class Plan:
    groups: list = field(default_factory=list)
    schedule: dict = field(default_factory=dict)  # logN -> bounds


class BatchRunner:
    """Plans, packs and runs a mixed batch; optionally as one CUDA graph."""

    def __init__(self, contexts: dict, k: int):
        self.ctx = contexts  # logN -> Context (keys resident)
        self.k = int(k)
        import torch

        self.torch = torch
        self.graph = None

    def plan(self, items: list[Item], schedule: dict) -> Plan:
        torch = self.torch
        plan = Plan(schedule=dict(schedule))
        by_ring = {}
        for i, it in enumerate(items):
            by_ring.setdefault(it.logN, []).append(i)
        for logN, idx in sorted(by_ring.items()):
            bounds = schedule[logN]
            lo = -1
            for hi in bounds:
                members = [i for i in idx if lo < items[i].logQ <= hi]
                lo = hi
                if not members:
                    continue
                logQ_max = max(items[i].logQ for i in members)
                ctx = self.ctx[logN]
                L_pad = limbs(logQ_max)
                n = len(members)
                N = 1 << logN
                g = Group(ctx, logN, members, logQ_max, L_pad)
                g.A = torch.zeros((n, 2, L_pad, N), dtype=torch.int32, device=ctx.device)
                g.B = torch.zeros_like(g.A)
                g.O = torch.zeros_like(g.A)
                g.bits = torch.tensor([items[i].logQ for i in members], dtype=torch.int32, device=ctx.device)
                plan.groups.append(g)
        return plan

    def pack(self, plan: Plan, items: list[Item]) -> None:
        for g in plan.groups:
            for j, i in enumerate(g.idx):
                L = items[i].a.data.shape[2]
                g.A[j, :, :L].copy_(items[i].a.data[0])
                g.B[j, :, :L].copy_(items[i].b.data[0])

    def run(self, plan: Plan) -> None:
        for g in plan.groups:
            fhe_mult_relin_rescale_ragged(g.ctx, g.A, g.B, g.O, g.bits, g.logQ_max, self.k)

    def capture(self, plan: Plan):
        """Capture run(plan) into a CUDA graph (workspaces are sized by a first eager run)."""
        torch = self.torch
        self.run(plan)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run(plan)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = g
        return g

    def outputs(self, plan: Plan, items: list[Item]) -> list:
        """Per item: (2, L_out, N) result tensor views at modulus 2^(logQ - k)."""
        out = [None] * len(items)
        for g in plan.groups:
            for j, i in enumerate(g.idx):
                out[i] = g.O[j, :, :limbs(items[i].logQ - self.k)].contiguous()
        return out

    def per_op(self, items: list[Item]) -> list:
        """The plain path: one fhe_mult_relin_rescale call per pair (cnum = 1)."""
        res = []
        for it in items:
            ctx = self.ctx[it.logN]
            o = ctx.empty_ct(1, it.logQ - self.k)
            fhe_mult_relin_rescale(ctx, it.a, it.b, self.k, o)
            res.append(o)
        return res


class Autotuner:
    """Chooses the level-bucket count per ring size by measuring candidate plans; caches the choice."""

    CANDIDATES = (1, 2, 4, 8, 12, 16)

    def __init__(self, cache_path: str | None = None):
        self.cache_path = cache_path
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                self.cache = json.load(open(cache_path))
            except (OSError, ValueError):
                self.cache = {}

    @staticmethod
    def key(gpu: str, logN: int, n: int) -> str:
        size_class = 1 << max(0, int(np.ceil(np.log2(max(1, n)))))
        return f"{gpu}|N=2^{logN}|n<={size_class}"

    def tune(self, runner: BatchRunner, items: list[Item], reps: int = 2) -> dict:
        torch = runner.torch
        gpu = torch.cuda.get_device_name()
        by_ring = {}
        for it in items:
            by_ring.setdefault(it.logN, []).append(it.logQ)
        schedule, report = {}, {}
        for logN, levels in sorted(by_ring.items()):
            key = self.key(gpu, logN, len(levels))
            sub = [it for it in items if it.logN == logN]
            if key in self.cache:
                nb = int(self.cache[key])
            else:
                best = None
                timings = {}
                for nb in self.CANDIDATES:
                    sched = {logN: bucket_bounds(levels, nb)}
                    plan = runner.plan(sub, sched)
                    runner.pack(plan, sub)
                    runner.run(plan)  # warm / size workspaces
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        runner.run(plan)
                    e1.record()
                    e1.synchronize()
                    timings[nb] = e0.elapsed_time(e1) / reps
                    if best is None or timings[nb] < timings[best]:
                        best = nb
                    del plan
                nb = best
                self.cache[key] = nb
                report[logN] = timings
            schedule[logN] = bucket_bounds(levels, nb)
        if self.cache_path:
            try:
                json.dump(self.cache, open(self.cache_path, "w"), indent=1)
            except OSError:
                pass
        return {"schedule": schedule, "timings_ms": report}
