"""Continuous-batching request server for homomorphic mult / rotate / degree-7 polynomial requests.

Keys and ciphertext state stay resident in HBM.  Requests arrive over time
(Poisson arrivals in the benchmark) and carry a level (modulus 2^logQ).  The
serving loop:

* admits arrived requests while the device-memory footprint of admitted work
  (outputs, intermediates and workspace share at the request's level) stays
  within a budget;
* forms batches from everything admitted and ready: multiplications go into
  ragged batches (`fhe_mult_relin_rescale_ragged`, each ciphertext keeps its
  own modulus), rotations into batches of one (step, level);
* keeps several batches in flight on separate CUDA streams, so requests that
  arrive while others run are admitted as memory and streams free up and
  their work overlaps on the device;
* advances multi-stage requests (the polynomial) stage by stage and records
  arrival-to-completion latency; a request's final limb work runs on its own
  stream and completes by event, so the loop never waits on the device.

Multiplications are grouped by limb count (levels within 32 bits of each
other), so a batch pays for at most one limb of padding, and rotations by
(step, level).  Failures are handled on the host: a completion callback that
raises marks only its own request, and a batch whose stream reports an error
(`fail_batch`, a hook tests use to inject one) fails only its own requests;
the server finishes the rest.

`run_per_op` serves the same request stream without batching: each request,
as it arrives, is issued alone through the plain calls on one stream (the
baseline the served form is measured against).  When a request arrives to an
idle server it runs whole on one stream (`whole_request`), its polynomial's
independent products two at a time.

Results are exact: a request's ciphertext is the same, bit for bit, whether it
ran alone or inside any mix (the ragged batch uses the widest member's primes,
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
    error: str = ""


@dataclass
class Task:
    """One primitive of a request stage: a multiplication or a rotation."""

    req: Request
    kind: str               # "mult" | "rotate" | "whole" (the request run alone)
    name: str               # register written
    x: object = None        # operand tensors (2, L, N) views
    y: object = None
    logQ: int = 0
    step: int = 0


def linear_part(ctx: Context, terms: dict, l3: int, k: int):
    """sum_i C_i x^i + C_0 2^k at level l3, then rescale by COEF_SHIFT bits (on the current stream)."""
    acc = None
    for i, t in terms.items():
        o = ctx.empty_ct(1, l3)
        fhe_mult_const(ctx, Ciphertext(t.unsqueeze(0), l3), COEF_2_30[i], o)
        if acc is None:
            acc = o
        else:
            fhe_add(ctx, acc, o, acc)
    fhe_add_const(ctx, acc, COEF_2_30[0], k, acc)
    out = ctx.empty_ct(1, l3 - COEF_SHIFT)
    fhe_rescale(ctx, acc, COEF_SHIFT, out)
    return out.data[0]


class Server:
    def __init__(self, ctx: Context, pool: dict, k: int, budget_bytes: int, max_batch: int = 64, streams: int = 2,
                 fail_batch=None):
        import torch

        self.torch = torch
        self.ctx = ctx
        self.pool = pool            # logQ -> Ciphertext batch (cnum_pool, 2, L, N)
        self.k = int(k)
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.streams = [torch.cuda.Stream() for _ in range(max(1, streams))]
        self.finish_stream = torch.cuda.Stream()
        self.ws = [None] * len(self.streams)
        self.busy = [None] * len(self.streams)   # (event, tasks, outputs) per stream
        self.fail_batch = fail_batch              # (stream index, tasks) -> True to fail that batch (injection)
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
        """Linear combination at level l - 3k on the finishing stream; returns the event that completes it."""
        torch = self.torch
        k, l3 = self.k, r.logQ - 3 * self.k
        fs_ = self.finish_stream
        fs_.wait_stream(torch.cuda.current_stream())  # the mod-downs of the operands run on the main stream
        with torch.cuda.stream(fs_):
            x = self._operand(r, r.a)
            terms = {1: self._down(x, r.logQ, l3, r, "x_d3"),
                     3: self._down(r.regs["x3"], r.logQ - 2 * k, l3, r, "x3_d"), 5: r.regs["x5"], 7: r.regs["x7"]}
            for t in terms.values():
                t.record_stream(fs_)
            r.result = linear_part(self.ctx, terms, l3, k)
            ev = torch.cuda.Event()
            ev.record(fs_)
        r.result.record_stream(torch.cuda.current_stream())
        return ev

    def _advance(self, r: Request, now: float):
        """Called when the request's stage tasks are done: True if the request is complete, an event
        if its final work is in flight, False if another stage follows."""
        if r.op in ("mult", "rotate"):
            r.result = r.regs["out"]
            return True
        r.stage += 1
        if r.stage == 3:
            return self._finish_poly(r)
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
                # one limb count per batch: canonical operands are zero above their own level already
                lq_max = max(t.logQ for t in tasks)
                n = len(tasks)
                A = torch.stack([t.x for t in tasks])
                B = torch.stack([t.y for t in tasks])
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

    def _solo(self, ready: list):
        """The request to run whole when the ready work is one request at its first stage and every
        stream is idle (at low load nothing would join its batches), else None."""
        if any(b is not None for b in self.busy):
            return None
        req = ready[0].req
        if req.stage != 0 or any(t.req is not req for t in ready):
            return None
        return req

    def _launch_whole(self, si: int, req: Request):
        """All of the request's work on stream si, one event at the end (whole_request: the plain calls,
        the polynomial's independent products two at a time)."""
        torch = self.torch
        st = self.streams[si]
        st.wait_stream(torch.cuda.current_stream())
        self._pending_ready_drop(req)
        with torch.cuda.stream(st):
            out = whole_request(self.ctx, self.pool, req, self.k)
            ev = torch.cuda.Event()
            ev.record(st)
        self.busy[si] = (ev, [Task(req, "whole", "out")], [out])

    def _pending_ready_drop(self, req: Request):
        self._ready_ref[:] = [t for t in self._ready_ref if t.req is not req]

    def _pick_batch(self, ready: list) -> list:
        """Tasks of one kind from the oldest ready request: mults of any level, rotations of one (step, level)."""
        if not ready:
            return []
        first = ready[0]
        if first.kind == "mult":
            nl = limbs(first.logQ)
            sel = [t for t in ready if t.kind == "mult" and limbs(t.logQ) == nl][: self.max_batch]
        else:
            sel = [t for t in ready if t.kind == "rotate" and t.step == first.step and t.logQ == first.logQ]
            sel = sel[: self.max_batch]
        ids = set(map(id, sel))
        ready[:] = [t for t in ready if id(t) not in ids]
        return sel

    # ------------------------------------------------------------------- loop
    def run(self, requests: list, time_scale: float = 1.0, max_wall_s: float = 1e9, on_done=None) -> dict:
        """Serve `requests` (arrival times in seconds); on_done(request) is called for each completed request."""
        torch = self.torch
        arrivals = deque(sorted(requests, key=lambda r: r.t_arrive))
        queue = deque()
        ready = []
        self._ready_ref = ready
        waiting = {}   # request id -> number of outstanding tasks
        finishing = deque()  # (event, request): final limb work in flight
        failed_ids = set()
        in_use = 0
        done, failed = [], []
        cb_errors = 0
        t0 = time.perf_counter()
        torch.cuda.synchronize()

        def complete(req, tnow):
            nonlocal in_use, cb_errors
            req.t_done = tnow
            in_use -= req.footprint
            done.append(req)
            req.regs = {}
            if on_done is not None:
                try:
                    on_done(req)
                except Exception as exc:  # a failing callback marks its own request only
                    req.error = f"callback: {exc!r}"
                    cb_errors += 1

        while len(done) + len(failed) < len(requests):
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
            while finishing and finishing[0][0].query():
                _, req = finishing.popleft()
                complete(req, (time.perf_counter() - t0) / time_scale)
                progressed = True
            for si in range(len(self.streams)):
                b = self.busy[si]
                if b is not None and b[0].query():
                    self.busy[si] = None
                    progressed = True
                    bad = self.fail_batch is not None and self.fail_batch(si, b[1])
                    if b[1] and b[1][0].kind == "whole":  # a request that ran whole on this stream
                        req = b[1][0].req
                        if bad:
                            req.error = f"stream {si} reported an error"
                            failed_ids.add(req.rid)
                            in_use -= req.footprint
                            failed.append(req)
                        else:
                            req.result = b[2][0]
                            req.result.record_stream(torch.cuda.current_stream())
                            complete(req, (time.perf_counter() - t0) / time_scale)
                        continue
                    for t, o in zip(b[1], b[2]):
                        req = t.req
                        if req.rid in failed_ids:
                            continue
                        if bad:  # this batch's results are lost: fail its requests, keep serving the others
                            req.error = f"stream {si} reported an error"
                            failed_ids.add(req.rid)
                            in_use -= req.footprint
                            req.regs = {}
                            failed.append(req)
                            continue
                        o.record_stream(torch.cuda.current_stream())  # consumed on the main stream from here on
                        req.regs[t.name] = o
                        waiting[req.rid] -= 1
                        if waiting[req.rid] == 0:
                            adv = self._advance(req, (time.perf_counter() - t0) / time_scale)
                            if adv is True:
                                complete(req, (time.perf_counter() - t0) / time_scale)
                            elif adv is False:
                                tasks = self._stage_tasks(req)
                                waiting[req.rid] = len(tasks)
                                ready.extend(tasks)
                            else:
                                finishing.append((adv, req))
            if failed_ids:
                ready[:] = [t for t in ready if t.req.rid not in failed_ids]
            for si in range(len(self.streams)):
                if self.busy[si] is None and ready:
                    solo = self._solo(ready)
                    if solo is not None:  # nothing to batch with: run the whole request on this stream
                        self._launch_whole(si, solo)
                        progressed = True
                        continue
                    batch = self._pick_batch(ready)
                    if batch:
                        self._launch(si, batch)
                        progressed = True
            if not progressed:
                in_flight = finishing or any(b is not None for b in self.busy)
                if not in_flight:  # idle: sleep until the next arrival (at most 1 ms)
                    nxt = arrivals[0].t_arrive * time_scale if arrivals else now * time_scale + 0.001
                    time.sleep(min(max(nxt - (time.perf_counter() - t0), 0.0), 0.001))
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / time_scale
        return _stats(done, len(requests), wall, failed=len(failed), callback_errors=cb_errors)


def _stats(done: list, offered: int, wall: float, **extra) -> dict:
    lat = np.array([r.t_done - r.t_arrive for r in done]) * 1e3
    out = {"completed": len(done), "offered": offered, "wall_s": wall,
           "ops_per_s": len(done) / wall if wall > 0 else 0.0,
           "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
           "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
           "by_op": {op: int(sum(1 for r in done if r.op == op)) for op in ("mult", "rotate", "poly7")}}
    out.update(extra)
    return out


def per_op_request(ctx: Context, pool: dict, r: Request, k: int):
    """One request alone through the plain calls (cnum 1) on the current stream; returns its result tensor."""
    x = Ciphertext(pool[r.logQ].data[r.a:r.a + 1], r.logQ)
    if r.op == "mult":
        y = Ciphertext(pool[r.logQ].data[r.b:r.b + 1], r.logQ)
        return ctx.mult_relin_rescale(x, y, k).data[0]
    if r.op == "rotate":
        return ctx.rotate(x, r.step).data[0]
    l0 = r.logQ
    x2 = ctx.mult_relin_rescale(x, x, k)
    x3 = ctx.mult_relin_rescale(x2, ctx.moddown(x, l0 - k), k)
    x4 = ctx.mult_relin_rescale(x2, x2, k)
    x5 = ctx.mult_relin_rescale(x4, ctx.moddown(x, l0 - 2 * k), k)
    x7 = ctx.mult_relin_rescale(x4, x3, k)
    l3 = l0 - 3 * k
    terms = {1: ctx.moddown(x, l3).data[0], 3: ctx.moddown(x3, l3).data[0], 5: x5.data[0], 7: x7.data[0]}
    return linear_part(ctx, terms, l3, k)


def whole_request(ctx: Context, pool: dict, r: Request, k: int):
    """One request alone on the current stream, its independent products batched: the polynomial's x3 and
    x4 (both at level l - k) run as one CipherTensor of two, and so do x5 and x7 (level l - 2k), so its
    critical path is three multiplications instead of five.  Every ciphertext equals per_op_request's."""
    import torch

    if r.op != "poly7":
        return per_op_request(ctx, pool, r, k)
    x = Ciphertext(pool[r.logQ].data[r.a:r.a + 1], r.logQ)
    l0 = r.logQ
    x2 = ctx.mult_relin_rescale(x, x, k)
    xd1 = ctx.moddown(x, l0 - k)
    p1 = ctx.mult_relin_rescale(Ciphertext(torch.cat([x2.data, x2.data]), l0 - k),
                                Ciphertext(torch.cat([xd1.data, x2.data]), l0 - k), k)  # x3, x4
    x3, x4 = p1.data[0:1], p1.data[1:2]
    xd2 = ctx.moddown(x, l0 - 2 * k)
    p2 = ctx.mult_relin_rescale(Ciphertext(torch.cat([x4, x4]), l0 - 2 * k),
                                Ciphertext(torch.cat([xd2.data, x3]), l0 - 2 * k), k)  # x5, x7
    l3 = l0 - 3 * k
    terms = {1: ctx.moddown(x, l3).data[0], 3: ctx.moddown(Ciphertext(x3, l0 - 2 * k), l3).data[0],
             5: p2.data[0], 7: p2.data[1]}
    return linear_part(ctx, terms, l3, k)


def run_per_op(ctx: Context, pool: dict, requests: list, k: int, time_scale: float = 1.0, on_done=None,
               max_outstanding: int = 256) -> dict:
    """The same request stream without batching: each request, as it arrives, issued alone through the
    plain calls on the current stream (at most max_outstanding in flight); completion by one event per
    request; on_done(request) after each completion."""
    import torch

    reqs = sorted(requests, key=lambda r: r.t_arrive)
    outstanding = deque()
    done = []
    i = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while len(done) < len(reqs):
        now = (time.perf_counter() - t0) / time_scale
        progressed = False
        while i < len(reqs) and reqs[i].t_arrive <= now and len(outstanding) < max_outstanding:
            r = reqs[i]
            i += 1
            r.result = per_op_request(ctx, pool, r, k)
            ev = torch.cuda.Event()
            ev.record()
            outstanding.append((ev, r))
            progressed = True
        while outstanding and outstanding[0][0].query():
            _, r = outstanding.popleft()
            r.t_done = (time.perf_counter() - t0) / time_scale
            done.append(r)
            if on_done is not None:
                on_done(r)
            progressed = True
        if not progressed:
            time.sleep(0.0002)
    torch.cuda.synchronize()
    return _stats(done, len(reqs), (time.perf_counter() - t0) / time_scale)


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
