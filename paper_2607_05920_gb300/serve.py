"""Continuous-batching request server for homomorphic mult / rotate / degree-7 polynomial requests.

Keys and ciphertext state stay resident in HBM.  Requests arrive over time
(Poisson arrivals in the benchmark) and carry a level (modulus 2^logQ).  The
serving loop:

* admits arrived requests while the device-memory footprint of admitted work
  (outputs, intermediates and workspace share at the request's level) stays
  within a budget;
* forms batches from everything admitted and ready: multiplications of any
  level go into one ragged batch (`fhe_mult_relin_rescale_ragged`, each
  ciphertext keeps its own modulus), rotations are grouped by (step, level);
* keeps several batches in flight on separate CUDA streams, so requests that
  arrive while others run are admitted as memory and streams free up and
  their work overlaps on the device;
* advances multi-stage requests (the polynomial) stage by stage and records
  arrival-to-completion latency.

Results are exact: a request's ciphertext is the same, bit for bit, whether it
ran alone or inside any mix (the ragged batch uses the widest level's primes,
which is exact for every member).

The degree-7 request evaluates an odd sigmoid-like polynomial fitted once by
FP64 least squares to 1/(1+e^-x) on [-8, 8]: p(x) = c0 + c1 x + c3 x^3 + c5 x^5
+ c7 x^7 with c scaled by 2^30 to integers (COEF_2_30), using the products
x2 = x x, x3 = x2 x, x4 = x2 x2, x5 = x4 x, x7 = x4 x3 (depth 3, rescale by
the scale bits after each), integer constant multiplications, additions and
a final rescale by 30 bits.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import (FHE_OP_MULT_RAGGED, FHE_OP_ROTATE, Ciphertext, Context, fhe_add, fhe_add_const,
               fhe_moddown, fhe_mult_const, fhe_mult_relin_rescale_ragged, fhe_rescale, fhe_rotate, lib, limbs)

# c0, c1, c3, c5, c7 of the fit, times 2^30, rounded
COEF_SHIFT = 30
COEF_2_30 = {0: 536870912, 1: 232868762, 3: -8795410, 5: 178024, 7: -1283}


@dataclass
class Request:
    rid: int
    t_arrive: float
    op: str                 # "mult" | "rotate" | "poly7"
    logQ: int
    a: int                  # index into the level's resident pool
    b: int = 0
    step: int = 0
    stage: int = 0
    regs: dict = field(default_factory=dict)
    t_admit: float = -1.0
    t_done: float = -1.0
    result: object = None
    footprint: int = 0


@dataclass
class Task:
    """One primitive of a request stage: a multiplication or a rotation."""

    req: Request
    kind: str               # "mult" | "rotate"
    name: str               # register written
    x: object = None        # operand tensors (2, L, N) views
    y: object = None
    logQ: int = 0
    step: int = 0


class Server:
    def __init__(self, ctx: Context, pool: dict, k: int, budget_bytes: int, max_batch: int = 64, streams: int = 2):
        import torch

        self.torch = torch
        self.ctx = ctx
        self.pool = pool            # logQ -> Ciphertext batch (cnum_pool, 2, L, N)
        self.k = int(k)
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.streams = [torch.cuda.Stream() for _ in range(max(1, streams))]
        self.ws = [None] * len(self.streams)
        self.busy = [None] * len(self.streams)   # (event, tasks, outputs) per stream
        self.N = ctx.N

    # ------------------------------------------------------------ footprints
    def ct_bytes(self, logQ: int, cnum: int = 1) -> int:
        return int(lib.fhe_ct_bytes(self.ctx.logN, int(logQ), int(cnum)))

    def footprint(self, r: Request) -> int:
        ws = int(lib.fhe_workspace_bytes(self.ctx.handle, FHE_OP_MULT_RAGGED, r.logQ, 1))
        if r.op == "poly7":
            return 9 * self.ct_bytes(r.logQ) + ws
        return 2 * self.ct_bytes(r.logQ) + ws

    # ----------------------------------------------------------- request flow
    def _operand(self, r: Request, which: int):
        return self.pool[r.logQ].data[which]

    def _ct(self, t, logQ):
        return Ciphertext(t.unsqueeze(0), logQ)

    def _stage_tasks(self, r: Request) -> list:
        """The batchable primitives of the request's current stage (after its cheap limb work)."""
        k = self.k
        if r.op == "mult":
            return [Task(r, "mult", "out", self._operand(r, r.a), self._operand(r, r.b), r.logQ)]
        if r.op == "rotate":
            return [Task(r, "rotate", "out", self._operand(r, r.a), None, r.logQ, r.step)]
        # poly7
        x = self._operand(r, r.a)
        l0 = r.logQ
        if r.stage == 0:
            return [Task(r, "mult", "x2", x, x, l0)]
        if r.stage == 1:
            xd = self._down(x, l0, l0 - k, r, "x_d1")
            return [Task(r, "mult", "x3", r.regs["x2"], xd, l0 - k), Task(r, "mult", "x4", r.regs["x2"],
                                                                          r.regs["x2"], l0 - k)]
        if r.stage == 2:
            xd2 = self._down(x, l0, l0 - 2 * k, r, "x_d2")
            return [Task(r, "mult", "x5", r.regs["x4"], xd2, l0 - 2 * k),
                    Task(r, "mult", "x7", r.regs["x4"], r.regs["x3"], l0 - 2 * k)]
        return []

    def _down(self, t, from_logQ, to_logQ, r, name):
        if name in r.regs and r.regs[name] is not None:
            return r.regs[name]
        out = self.ctx.empty_ct(1, to_logQ)
        fhe_moddown(self.ctx, self._ct(t, from_logQ), out)
        r.regs[name] = out.data[0]
        return r.regs[name]

    def _finish_poly(self, r: Request):
        """Linear combination at level l - 3k: sum C_i x^i + C_0 Delta, then rescale by 30 bits."""
        k, l3 = self.k, r.logQ - 3 * self.k
        x = self._operand(r, r.a)
        terms = {1: self._down(x, r.logQ, l3, r, "x_d3"), 3: self._down(r.regs["x3"], r.logQ - 2 * k, l3, r, "x3_d"),
                 5: r.regs["x5"], 7: r.regs["x7"]}
        acc = None
        for i, t in terms.items():
            o = self.ctx.empty_ct(1, l3)
            fhe_mult_const(self.ctx, self._ct(t, l3), COEF_2_30[i], o)
            if acc is None:
                acc = o
            else:
                fhe_add(self.ctx, acc, o, acc)
        fhe_add_const(self.ctx, acc, COEF_2_30[0], k, acc)
        out = self.ctx.empty_ct(1, l3 - COEF_SHIFT)
        fhe_rescale(self.ctx, acc, COEF_SHIFT, out)
        return out.data[0]

    def _advance(self, r: Request, now: float) -> bool:
        """Called when the request's stage tasks are done; True if the request is complete."""
        if r.op in ("mult", "rotate"):
            r.result = r.regs["out"]
            return True
        r.stage += 1
        if r.stage == 3:
            r.result = self._finish_poly(r)
            return True
        return False

    # ----------------------------------------------------------------- batches
    def _launch(self, si: int, tasks: list):
        torch = self.torch
        st = self.streams[si]
        main = torch.cuda.current_stream()
        st.wait_stream(main)  # operands prepared on the main stream (mod-downs) come first
        for t in tasks:       # keep operand memory alive for this stream's reads
            for v in (t.x, t.y):
                if v is not None:
                    v.record_stream(st)
        with torch.cuda.stream(st):
            if tasks[0].kind == "mult":
                lq_max = max(t.logQ for t in tasks)
                L_pad = limbs(lq_max)
                n = len(tasks)
                A = torch.zeros((n, 2, L_pad, self.N), dtype=torch.int32, device=self.ctx.device)
                B = torch.zeros_like(A)
                for j, t in enumerate(tasks):
                    A[j, :, :t.x.shape[1]].copy_(t.x)
                    B[j, :, :t.y.shape[1]].copy_(t.y)
                O = torch.empty_like(A)
                bits = torch.tensor([t.logQ for t in tasks], dtype=torch.int32, device=self.ctx.device)
                need = int(lib.fhe_workspace_bytes(self.ctx.handle, FHE_OP_MULT_RAGGED, lq_max, n))
                if self.ws[si] is None or self.ws[si].numel() < need:
                    self.ws[si] = torch.empty(need, dtype=torch.uint8, device=self.ctx.device)
                fhe_mult_relin_rescale_ragged(self.ctx, A, B, O, bits, lq_max, self.k, ws=self.ws[si])
                outs = [O[j, :, :limbs(t.logQ - self.k)].contiguous() for j, t in enumerate(tasks)]
            else:
                lq, step = tasks[0].logQ, tasks[0].step
                X = torch.stack([t.x for t in tasks])
                out = self.ctx.empty_ct(len(tasks), lq)
                need = int(lib.fhe_workspace_bytes(self.ctx.handle, FHE_OP_ROTATE, lq, len(tasks)))
                if self.ws[si] is None or self.ws[si].numel() < need:
                    self.ws[si] = torch.empty(need, dtype=torch.uint8, device=self.ctx.device)
                fhe_rotate(self.ctx, Ciphertext(X, lq), step, out, ws=self.ws[si])
                outs = [out.data[j] for j in range(len(tasks))]
            ev = torch.cuda.Event()
            ev.record(st)
        self.busy[si] = (ev, tasks, outs)

    def _pick_batch(self, ready: list) -> list:
        """Tasks of one kind from the oldest ready request: mults of any level, rotations of one (step, level)."""
        if not ready:
            return []
        first = ready[0]
        if first.kind == "mult":
            sel = [t for t in ready if t.kind == "mult"][: self.max_batch]
        else:
            sel = [t for t in ready if t.kind == "rotate" and t.step == first.step and t.logQ == first.logQ]
            sel = sel[: self.max_batch]
        ids = set(map(id, sel))
        ready[:] = [t for t in ready if id(t) not in ids]
        return sel

    # ------------------------------------------------------------------- loop
    def run(self, requests: list, time_scale: float = 1.0, max_wall_s: float = 1e9) -> dict:
        torch = self.torch
        arrivals = deque(sorted(requests, key=lambda r: r.t_arrive))
        queue = deque()
        ready = []
        waiting = {}   # request id -> number of outstanding tasks
        in_use = 0
        done = []
        t0 = time.perf_counter()
        torch.cuda.synchronize()
        while len(done) < len(requests):
            now = (time.perf_counter() - t0) / time_scale
            if now * time_scale > max_wall_s:
                break
            while arrivals and arrivals[0].t_arrive <= now:
                queue.append(arrivals.popleft())
            while queue:
                r = queue[0]
                fp = self.footprint(r)
                if in_use + fp > self.budget and in_use > 0:
                    break
                queue.popleft()
                r.footprint = fp
                in_use += fp
                r.t_admit = now
                tasks = self._stage_tasks(r)
                waiting[r.rid] = len(tasks)
                ready.extend(tasks)
            progressed = False
            for si in range(len(self.streams)):
                b = self.busy[si]
                if b is not None and b[0].query():
                    self.busy[si] = None
                    progressed = True
                    for t, o in zip(b[1], b[2]):
                        o.record_stream(torch.cuda.current_stream())  # consumed on the main stream from here on
                        t.req.regs[t.name] = o
                        waiting[t.req.rid] -= 1
                        if waiting[t.req.rid] == 0:
                            tnow = (time.perf_counter() - t0) / time_scale
                            if self._advance(t.req, tnow):
                                if t.req.op == "poly7":  # its final limb work ran on the main stream
                                    torch.cuda.current_stream().synchronize()
                                    tnow = (time.perf_counter() - t0) / time_scale
                                t.req.t_done = tnow
                                in_use -= t.req.footprint
                                done.append(t.req)
                                t.req.regs = {}
                            else:
                                tasks = self._stage_tasks(t.req)
                                waiting[t.req.rid] = len(tasks)
                                ready.extend(tasks)
            for si in range(len(self.streams)):
                if self.busy[si] is None and ready:
                    batch = self._pick_batch(ready)
                    if batch:
                        self._launch(si, batch)
                        progressed = True
            if not progressed:
                time.sleep(0.0002)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / time_scale
        lat = np.array([r.t_done - r.t_arrive for r in done]) * 1e3
        return {"completed": len(done), "offered": len(requests), "wall_s": wall,
                "ops_per_s": len(done) / wall if wall > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "by_op": {op: int(sum(1 for r in done if r.op == op)) for op in ("mult", "rotate", "poly7")}}


def make_requests(g, rate_hz: float, duration_s: float, levels: list, pool_size: int, steps: list,
                  mix=(0.5, 0.3, 0.2)) -> list:
    """Poisson arrivals; op mix mult/rotate/poly7; level, operands and rotation step drawn from the seed."""
    from fhe_synth import poisson_arrivals

    times = poisson_arrivals(g, rate_hz, duration_s)
    ops = g.choice(["mult", "rotate", "poly7"], size=len(times), p=list(mix))
    reqs = []
    for i, (t, op) in enumerate(zip(times, ops)):
        lq = int(levels[int(g.integers(0, len(levels)))])
        reqs.append(Request(i, float(t), str(op), lq, int(g.integers(0, pool_size)), int(g.integers(0, pool_size)),
                            int(steps[int(g.integers(0, len(steps)))])))
    return reqs
