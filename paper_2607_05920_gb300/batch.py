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
`Autotuner` searches three levels of schedule on the batch at hand: the bucket
count per ring size, then for every group the kernel forms of its ring
products (tensor-core or integer reconstruction, tensor-core or integer lift,
fused or split transform schedule; `fhe_set_forms`), and keeps the fastest,
cached per (GPU, ring size, limb count, batch size class), and finally whether
the ring sizes run one after another or as parallel graph branches (one
stream per ring size).  Every form gives bit-identical results, so the choice
is a pure schedule.

All arithmetic runs in the library's kernels; this module only plans, packs
(device-to-device copies into padded tensors) and launches.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

from . import (FHE_CRT_DIRECT, FHE_CRT_DIRECT_INT, FHE_LIFT_AUTO, FHE_LIFT_INT, FHE_LIFT_TC, FHE_NTT_FUSED,
               FHE_NTT_FUSED_GROUPS, FHE_NTT_SPLIT, FHE_OP_MULT_RAGGED, Ciphertext, Context, fhe_mult_relin_rescale,
               fhe_mult_relin_rescale_batch, fhe_mult_relin_rescale_ragged, fhe_set_forms, lib, limbs)

# (reconstruction, lift, transform schedule) candidates of a group
FORMS = tuple((c, l, t) for c in (FHE_CRT_DIRECT, FHE_CRT_DIRECT_INT) for l in (FHE_LIFT_TC, FHE_LIFT_INT)
              for t in (FHE_NTT_FUSED, FHE_NTT_FUSED_GROUPS, FHE_NTT_SPLIT))
DEFAULT_FORMS = (FHE_CRT_DIRECT, FHE_LIFT_AUTO, FHE_NTT_FUSED)
# work-table schedules (col_ctas_per_sm, row_ctas_per_sm, col_unit_rows): 0 CTAs per SM = one CTA per unit
TABLE_SCHEDS = tuple((c, r, u) for c in (0, 2, 3) for r in (0, 2, 4) for u in ((1,) if c == 0 else (1, 4, 16)))


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
    forms: tuple = DEFAULT_FORMS
    ws: object = None  # the group's own workspace on the work-table path


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
        self.branches = False  # ring sizes on parallel streams (graph branches); chosen by Autotuner
        self.table = None      # a work-table schedule: all groups in one fhe_mult_relin_rescale_batch call
        self.table_per_ring = False  # with a schedule: one call per ring size, rings as parallel branches
        self._streams = {}

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

    def run_group(self, g: Group, forms=None) -> None:
        fhe_set_forms(g.ctx, *(forms or g.forms))
        fhe_mult_relin_rescale_ragged(g.ctx, g.A, g.B, g.O, g.bits, g.logQ_max, self.k)

    def branch_streams(self, plan: Plan) -> dict:
        """One side stream per ring size of the plan (kept, so workspaces sized by an eager run are reused)."""
        torch = self.torch
        for logN in sorted({g.logN for g in plan.groups}):
            if logN not in self._streams:
                self._streams[logN] = torch.cuda.Stream()
        return self._streams

    def group_ws(self, g: Group):
        """The group's own workspace (the work-table call keeps every group's intermediates at once)."""
        nbytes = lib.fhe_workspace_bytes(g.ctx.handle, FHE_OP_MULT_RAGGED, int(g.logQ_max), len(g.idx))
        if g.ws is None or g.ws.numel() < nbytes:
            g.ws = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=g.ctx.device)
        return g.ws

    def run_table(self, plan: Plan, sched, per_ring: bool = False) -> None:
        """Every group in one fhe_mult_relin_rescale_batch call: lifts and reconstructions per group (default
        forms), each transform stage of all groups as one work-table launch with schedule `sched`.  With
        per_ring, one call per ring size, each on that ring's own stream (forked from and joined to the
        current one, so a captured graph holds the rings as parallel branches)."""
        torch = self.torch
        for c in {id(g.ctx): g.ctx for g in plan.groups}.values():
            fhe_set_forms(c, *DEFAULT_FORMS)

        def call(gs):
            groups = [(g.ctx, g.A, g.B, g.O, g.bits, g.logQ_max, self.group_ws(g)) for g in gs]
            for i in range(0, len(groups), 32):  # at most 32 groups (table segments) per call
                fhe_mult_relin_rescale_batch(groups[i:i + 32], self.k, sched)

        if not per_ring:
            call(plan.groups)
            return
        main = torch.cuda.current_stream()
        streams = self.branch_streams(plan)
        used = sorted({g.logN for g in plan.groups})
        for logN in used:
            streams[logN].wait_stream(main)
        for logN in used:
            with torch.cuda.stream(streams[logN]):
                call([g for g in plan.groups if g.logN == logN])
        for logN in used:
            main.wait_stream(streams[logN])

    def run(self, plan: Plan, branches: bool | None = None) -> None:
        """Launch every group (one work-table call when self.table holds a schedule).  With branches, the groups of each ring size go to that ring's own stream
        (forked from and joined back to the current stream): rings then overlap on the GPU, and in a
        captured graph they are independent branches.  Groups of one ring stay in order on one stream,
        so each stream keeps its own workspace."""
        torch = self.torch
        if self.table is not None:
            self.run_table(plan, self.table, self.table_per_ring)
            return
        if branches is None:
            branches = self.branches
        if not branches:
            for g in plan.groups:
                self.run_group(g)
        else:
            main = torch.cuda.current_stream()
            streams = self.branch_streams(plan)
            used = sorted({g.logN for g in plan.groups})
            for logN in used:
                streams[logN].wait_stream(main)
            for g in plan.groups:
                with torch.cuda.stream(streams[g.logN]):
                    self.run_group(g)
            for logN in used:
                main.wait_stream(streams[logN])
        for c in {id(g.ctx): g.ctx for g in plan.groups}.values():
            fhe_set_forms(c, *DEFAULT_FORMS)

    def capture(self, plan: Plan, branches: bool | None = None):
        """Capture run(plan) into a CUDA graph (workspaces are sized by a first eager run)."""
        torch = self.torch
        if branches is not None:
            self.branches = bool(branches)
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

    def per_level(self, items: list[Item]) -> list:
        """CipherTensor calls without raggedness: one fhe_mult_relin_rescale per (ring, exact level) with all
        pairs of that level stacked (cnum = their count)."""
        torch = self.torch
        by = {}
        for i, it in enumerate(items):
            by.setdefault((it.logN, it.logQ), []).append(i)
        res = [None] * len(items)
        for (logN, logQ), idx in sorted(by.items()):
            ctx = self.ctx[logN]
            a = Ciphertext(torch.cat([items[i].a.data for i in idx]), logQ)
            b = Ciphertext(torch.cat([items[i].b.data for i in idx]), logQ)
            o = ctx.empty_ct(len(idx), logQ - self.k)
            fhe_mult_relin_rescale(ctx, a, b, self.k, o)
            for j, i in enumerate(idx):
                res[i] = o.data[j]
        return res

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

    @staticmethod
    def forms_key(gpu: str, g: Group) -> str:
        size_class = 1 << max(0, int(np.ceil(np.log2(max(1, len(g.idx))))))
        return f"{gpu}|N=2^{g.logN}|L={g.L_pad}|n<={size_class}|forms"

    def tune_forms(self, runner: BatchRunner, plan: Plan, reps: int = 2) -> dict:
        """Per group: time every kernel form, keep the fastest (cached); returns {group index: ms per form}."""
        torch = runner.torch
        gpu = torch.cuda.get_device_name()
        report = {}
        for gi, g in enumerate(plan.groups):
            key = self.forms_key(gpu, g)
            if key in self.cache:
                g.forms = tuple(self.cache[key])
                continue
            timings = {}
            for f in FORMS:
                runner.run_group(g, f)  # warm (and sizes the workspace)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    runner.run_group(g, f)
                e1.record()
                e1.synchronize()
                timings[f] = e0.elapsed_time(e1) / reps
            g.forms = min(timings, key=timings.get)
            self.cache[key] = list(g.forms)
            report[gi] = {"/".join(map(str, f)): round(t, 4) for f, t in timings.items()}
            fhe_set_forms(g.ctx, *DEFAULT_FORMS)
        self._save()
        return report

    @staticmethod
    def branches_key(gpu: str, plan: Plan) -> str:
        rings = ",".join(str(n) for n in sorted({g.logN for g in plan.groups}))
        size_class = 1 << max(0, int(np.ceil(np.log2(max(1, sum(len(g.idx) for g in plan.groups))))))
        return f"{gpu}|rings={rings}|n<={size_class}|branches"

    def tune_branches(self, runner: BatchRunner, plan: Plan, reps: int = 3) -> dict:
        """Captures the plan with the ring sizes in sequence and as parallel branches, replays both and
        keeps the faster (cached); returns {form: ms per replay}."""
        torch = runner.torch
        key = self.branches_key(torch.cuda.get_device_name(), plan)
        if key in self.cache:
            runner.branches = bool(self.cache[key])
            return {}
        timings = {}
        for br in (False, True):
            graph = runner.capture(plan, branches=br)
            graph.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                graph.replay()
            e1.record()
            e1.synchronize()
            timings["branches" if br else "sequence"] = e0.elapsed_time(e1) / reps
            del graph
            runner.graph = None
        runner.branches = timings["branches"] < timings["sequence"]
        self.cache[key] = runner.branches
        self._save()
        return timings

    @staticmethod
    def table_key(gpu: str, plan: Plan) -> str:
        return Autotuner.branches_key(gpu, plan).replace("|branches", "|table")

    def tune_table(self, runner: BatchRunner, plan: Plan, reps: int = 2) -> dict:
        """Times the work-table call under every schedule of TABLE_SCHEDS, then captures the best one and the
        per-group graph (in the form tune_branches chose) and keeps the faster as runner.table (a schedule,
        or None for the per-group graph); cached.  Returns {schedule or form: ms}."""
        torch = runner.torch
        key = self.table_key(torch.cuda.get_device_name(), plan)
        if key in self.cache:
            v = self.cache[key]
            runner.table = tuple(v[1:]) if v else None
            runner.table_per_ring = bool(v[0]) if v else False
            return {}
        timings = {}
        for per_ring in (False, True):
            for sc in TABLE_SCHEDS:
                runner.run_table(plan, sc, per_ring)  # warm (and sizes the workspaces)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    runner.run_table(plan, sc, per_ring)
                e1.record()
                e1.synchronize()
                timings[(per_ring,) + sc] = e0.elapsed_time(e1) / reps
        bestk = min(timings, key=timings.get)
        best, runner.table_per_ring = bestk[1:], bestk[0]
        report = {("table per ring " if k[0] else "table ") + "/".join(map(str, k[1:])): round(t, 4)
                  for k, t in timings.items()}
        graphs = {}
        for mode in (best, None):
            runner.table = mode
            graph = runner.capture(plan)
            graph.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                graph.replay()
            e1.record()
            e1.synchronize()
            graphs[mode] = e0.elapsed_time(e1) / reps
            del graph
            runner.graph = None
        runner.table = best if graphs[best] < graphs[None] else None
        runner.table_per_ring = bool(runner.table) and runner.table_per_ring
        report["graph table"] = round(graphs[best], 4)
        report["graph groups"] = round(graphs[None], 4)
        self.cache[key] = [int(runner.table_per_ring)] + list(runner.table) if runner.table else None
        self._save()
        return report

    def _save(self):
        if self.cache_path:
            try:
                json.dump(self.cache, open(self.cache_path, "w"), indent=1)
            except OSError:
                pass

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
        self._save()
        return {"schedule": schedule, "timings_ms": report}
