#!/usr/bin/env python3
"""HMult + relinearisation + rescale throughput of the non-RNS CKKS hot path on GB300.

Workload (one step): a CipherTensor of `cnum` ciphertext pairs at N = 2^16,
Q = 2^1200, P = 2^1200, scale 2^40 -> fhe_mult_relin_rescale (k = 40).
Inputs are fresh public-key encryptions of seeded synthetic plaintexts
(coefficients of an encoded message at scale 2^40), already resident in HBM.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on the
same workload instead (the reference arm; bounded sample per step).
"""
from __future__ import annotations

import argparse
import copy
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LOGN, LOGQ, LOGP, K_RESCALE = 16, 1200, 1200, 40
E2E_CHUNKS = 4  # sub-batches of the end-to-end step (copies of one overlap compute of another)
METRIC = "HMult+relin+rescale ciphertexts/s at N=2^16 logQ=1200 (1 GB300)"
WORKLOAD = "CKKS N=2^16 logQ=logP=1200 scale 2^40: HMult+relin+rescale of a CipherTensor of ciphertext pairs"
SM_COUNT, SM_MAX_MHZ, IMAD_SLOTS_PER_CLK = 152, 2070.0, 64  # GB300: SMs, max SM clock, IMAD-pipe lanes/SM/clk


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cnum", type=int, default=64, help="ciphertext pairs per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--latency-iters", type=int, default=30)
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end to end: timed steps (default: as many as --steps)")
    ap.add_argument("--e2e-sub-batches", type=int, default=E2E_CHUNKS,
                    help="end to end: sub-batches whose upload, compute and download overlap")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrivals per second")
    ap.add_argument("--duration", type=float, default=2.0, help="serving: seconds of arrivals")
    ap.add_argument("--workload", default="ns", choices=["ns", "batched", "serving", "rotations", "bgv"],
                    help="ns: the headline N=2^16 logQ=1200 batch; batched: 512 uneven pairs, graph vs per-op")
    ap.add_argument("--ntt", default="fused", choices=["fused", "groups", "split"],
                    help="transform schedule of the ring products (fhe_set_forms)")
    ap.add_argument("--crt", default="direct", choices=["direct", "garner", "int"],
                    help="RNS->limb reconstruction: exact CRT with rounded quotient (dense sum on the tensor "
                         "cores), Garner mixed radix, or the exact CRT on the integer pipe only")
    args = ap.parse_args()
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    return args


# ----------------------------------------------------------------- oracle side
def _oracle_worker_init(seed):
    global _ORACLE_STATE
    import fhe_synth as fs
    from oracle import bigint, ckks

    g = fs.rng(seed)
    N = 1 << LOGN
    prm = ckks.CkksParams(LOGN, LOGQ, LOGP)
    s = [int(x) for x in fs.ternary(g, (), N)]
    a = bigint.from_limbs(fs.uniform_limbs(g, (), N, LOGQ + LOGP))
    e = [int(x) for x in fs.gaussian(g, (), N)]
    evk = ckks.relin_key(prm, s, a, e)
    la = fs.uniform_limbs(g, (2,), N, LOGQ)
    lb = fs.uniform_limbs(g, (2,), N, LOGQ)
    ca = tuple(bigint.from_limbs(la[i]) for i in range(2))
    cb = tuple(bigint.from_limbs(lb[i]) for i in range(2))
    _ORACLE_STATE = (evk, ca, cb)


def _oracle_step(_):
    from oracle import ckks

    evk, ca, cb = _ORACLE_STATE
    t0 = time.perf_counter()
    ckks.rescale(ckks.mult(ca, cb, evk, LOGQ, LOGP), K_RESCALE, LOGQ)
    return time.perf_counter() - t0


def oracle_throughput(steps: int, warmup: int, workers: int):
    """Run warmup + timed oracle steps (one ciphertext pair each) on `workers` spawned processes."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_oracle_worker_init, initargs=(1234,)) as pool:
        if warmup > 0:
            pool.map(_oracle_step, range(min(warmup, workers)), chunksize=1)
        t0 = time.perf_counter()
        per = pool.map(_oracle_step, range(steps), chunksize=1)
        wall = time.perf_counter() - t0
    return steps / wall, wall, per


def max_over_ranks(ms: float, dist, device: str) -> float:
    """The job's time for a timed region: the slowest rank's (`dist` None: one process)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: int, steps: int, ms: float) -> float:
    """Whole-job units/s: every rank processes its own batch of units each step (weak scaling)."""
    return world * units_per_rank * steps / (ms / 1e3)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    workers = max(1, min(args.steps, cores))
    value, wall, per = oracle_throughput(args.steps, args.warmup, workers)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ct/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int (Python big integers)",
        "data": "synthetic", "config": {"workload": WORKLOAD, "cnum": 1, "logN": LOGN, "logQ": LOGQ, "logP": LOGP,
                                        "log_scale": K_RESCALE},
        "cpu_baseline": {"value": value, "unit": "ct/s", "cores": workers, "kind": "oracle",
                         "sample": f"{args.steps} ciphertext pairs, one per step, steps spread over {workers} "
                                   f"spawned processes (one pair per process at a time)"},
        "e2e": {"value": value, "unit": "ct/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "per_step_s": {"p50": statistics.median(per), "max": max(per)},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- roofline counting
def crt_slots_direct(r: int, out_limbs: int) -> int:
    """IMAD-pipe slots of one direct-CRT reconstruction (one coefficient), algorithmic count.

    r Shoup products y_i (4 slots each), r x W limb multiply-adds (mad.wide, 2
    slots), W multiply-adds for kappa M.
    """
    return 4 * r + 2 * r * out_limbs + 2 * out_limbs


def crt_slots(r: int, out_limbs: int) -> int:
    """IMAD-pipe slots of one Garner reconstruction (one coefficient), algorithmic count.

    digits: r(r-1)/2 Shoup products (mul.hi = 2 slots, two mul.lo = 2 slots -> 4);
    Horner: per step the running value's limbs (capped at the output width),
    one 32x32->64 multiply-add (mad.wide = 2 slots) each.
    """
    digits = 4 * r * (r - 1) // 2
    horner = 0
    for k in range(r - 2, -1, -1):
        act = min(out_limbs, (31 * (r - k) + 31) // 32)
        horner += 2 * act
    return digits + horner


def crt_flops_tc(r: int, out_limbs: int) -> int:
    """Tensor-core FLOPs of one direct-CRT reconstruction (one coefficient), algorithmic count.

    The dense sum over r + 1 terms (y_i and kappa) times out_limbs limbs, in
    byte digits: 4 (r + 1) x 4 out_limbs multiply-adds, 2 FLOPs each (no
    padding of K to 16 or of the output columns to 16 counted).
    """
    return 2 * 4 * (r + 1) * 4 * out_limbs


def lift_flops_tc(r: int, limbs: int) -> int:
    """Tensor-core FLOPs of one lift (one coefficient to r residues), algorithmic count.

    The limb bytes (4 L) against the four digits of r constants: 4L x 4r
    multiply-adds, 2 FLOPs each (no padding counted).
    """
    return 2 * 4 * limbs * 4 * r


TENSOR_CLASSES = {"direct": ("crt", "lift")}


def step_work(fhe, cnum: int, crt_mode: str) -> dict:
    """Algorithmic work per step, by kernel class: IMAD-pipe slots, or tensor FLOPs for the tensor-core forms."""
    cs = {"garner": crt_slots, "int": crt_slots_direct, "direct": crt_flops_tc}[crt_mode]
    N = 1 << LOGN
    L = (LOGQ + 31) // 32
    rt = fhe.fhe_primes_for_bound(LOGN + 2 * LOGQ + 1)
    rk = fhe.fhe_primes_for_bound(LOGN + LOGQ + LOGP + LOGQ)
    lq_relin = (LOGQ + LOGP + 31) // 32
    # N > 2^12: the column stages (log N - 8 of them) run in the NTT passes, the
    # 8 row stages of both directions and the products in the fused pass
    col_st = LOGN - 8 if LOGN > 12 else LOGN
    row_bfly = N // 2 * (LOGN - col_st)
    col_bfly = N // 2 * col_st
    pw = cnum * N * (3 * rt + 2 * rk) * 6
    return {
        "crt": cnum * N * (3 * cs(rt, L) + 2 * cs(rk, lq_relin)),
        "ntt_fwd": cnum * (4 * rt + rk) * col_bfly * 4,
        # the N^-1 2^32 scale of the inverse is folded into the reconstruction's first product
        "ntt_inv": cnum * (3 * rt + 2 * rk) * col_bfly * 4,
        "ntt_pw": cnum * (7 * rt + 3 * rk) * row_bfly * 4 + (pw if LOGN > 12 else 0),
        "lift": (cnum * N * (4 * lift_flops_tc(rt, L) + lift_flops_tc(rk, L)) if crt_mode == "direct"
                 else cnum * N * (4 * rt * L + rk * L) * 2),
        "pointwise": pw if LOGN <= 12 else 0,
        "primes": {"tensor": rt, "keyswitch": rk},
    }


def class_roofline(k: str, n: int, t_ms: float, work: dict, args, total_ms: float) -> dict:
    """Per kernel class: launches, time, share and (where algorithmic work is counted) its roofline fraction."""
    out = {"launches": n, "ms": t_ms, "share": t_ms / max(1e-9, total_ms)}
    if k in work and t_ms > 0:
        rate = work[k] * args.steps / (t_ms / 1e3) / 1e12
        if k in TENSOR_CLASSES.get(args.crt, ()):
            peak = measured_peaks().get("bf16_tflops_sustained") or 1700.0
            out.update({"bound": "tensor", "achieved": rate, "unit": "TFLOP/s", "frac": rate / peak})
        else:
            peak = SM_COUNT * IMAD_SLOTS_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12
            out.update({"bound": "alu", "achieved": rate, "unit": "Tslot/s", "frac": rate / peak})
    return out


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


# the source files that define each kernel class (its own .cu and the headers it includes)
KERNEL_SOURCES = {
    "ntt_pw": ("common.cuh", "k_ntt.cu"),
    "ntt_fwd": ("common.cuh", "k_ntt.cu"),
    "ntt_inv": ("common.cuh", "k_ntt.cu"),
    "crt": ("common.cuh", "k_crt.cu", "tc.cuh"),
    "lift": ("common.cuh", "k_lift.cu", "tc.cuh"),
}


def source_digest(kernel: str) -> str:
    """sha256 of the kernel class's source files in the listed order, first 16 hex digits."""
    import hashlib

    src = os.path.join(ROOT, "paper_2607_05920_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the kernel's current source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    digest = source_digest(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
            return float(parts[2])
    return None


# --------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import fhe_synth as fs
    import paper_2607_05920_gb300 as fhe

    cnum = args.cnum
    N = 1 << LOGN
    L = fhe.limbs(LOGQ)
    g = fs.rng(77 + rank)
    crt = {"garner": fhe.FHE_CRT_GARNER, "int": fhe.FHE_CRT_DIRECT_INT, "direct": fhe.FHE_CRT_DIRECT}[args.crt]
    ctx = fhe.Context(LOGN, LOGQ, LOGP, crt=crt)
    ntt_form = {"fused": fhe.FHE_NTT_FUSED, "groups": fhe.FHE_NTT_FUSED_GROUPS, "split": fhe.FHE_NTT_SPLIT}[args.ntt]
    fhe.fhe_set_forms(ctx, crt, fhe.FHE_LIFT_AUTO, ntt_form)
    ctx.keygen_inject(fs.ternary(g, (), N), fs.uniform_limbs(g, (), N, LOGQ), fs.gaussian(g, (), N),
               fs.uniform_limbs(g, (), N, LOGQ + LOGP), fs.gaussian(g, (), N))

    def dev(a):
        a = np.ascontiguousarray(a)
        if a.dtype == np.uint32:
            a = a.view(np.int32)
        return torch.from_numpy(a.copy()).cuda()

    def encrypt_batch():
        m = fs.small_signed(g, (cnum,), N, K_RESCALE + 1)  # encoded-message-sized coefficients
        # two's complement limbs of m mod 2^logQ (argument marshalling of signed int64 plaintexts)
        pt = np.zeros((cnum, L, N), dtype=np.uint32)
        mu = m.astype(np.uint64)
        pt[:, 0, :] = (mu & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        pt[:, 1, :] = (mu >> np.uint64(32)).astype(np.uint32)
        neg = m < 0
        top = LOGQ - 32 * (L - 1)
        for l in range(2, L):
            pt[:, l, :] = np.where(neg, np.uint32(0xFFFFFFFF if (l < L - 1 or top == 32) else (1 << top) - 1), 0)
        if top < 32:
            pt[:, L - 1, :] &= np.uint32((1 << top) - 1)
        return ctx.encrypt_inject(dev(pt), dev(fs.ternary(g, (cnum,), N)), dev(fs.gaussian(g, (cnum,), N)),
                           dev(fs.gaussian(g, (cnum,), N)))

    A, B = encrypt_batch(), encrypt_batch()
    out = ctx.empty_ct(cnum, LOGQ - K_RESCALE)
    ctx.workspace(fhe.FHE_OP_MULT, LOGQ, cnum)
    torch.cuda.synchronize()

    def step():
        fhe.fhe_mult_relin_rescale(ctx, A, B, K_RESCALE, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    fhe.fhe_profile_reset(ctx, True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = fhe.fhe_profile_read(ctx)
    fhe.fhe_profile_reset(ctx, False)
    ms = max_over_ranks(ms, dist, "cuda")
    if dist:
        dist.barrier()
    value = job_throughput(world, cnum, args.steps, ms)
    launches = sum(n for n, _ in prof.values())

    # end to end: pinned host inputs -> device, compute, result -> host, every step.  The batch
    # goes in E2E_CHUNKS sub-batches: one stream uploads, one computes (the public call), one
    # downloads, ordered by events, so a sub-batch's copies overlap another's compute while the
    # compute kernels themselves run one at a time.
    A_h = A.data.cpu().pin_memory()
    B_h = B.data.cpu().pin_memory()
    out_h = torch.empty(out.data.shape, dtype=torch.int32).pin_memory()
    nchunk = args.e2e_sub_batches if cnum % args.e2e_sub_batches == 0 else 1
    per = cnum // nchunk
    up, comp, down = (torch.cuda.Stream() for _ in range(3))
    parts = [(fhe.Ciphertext(A.data[c * per:(c + 1) * per], LOGQ), fhe.Ciphertext(B.data[c * per:(c + 1) * per], LOGQ),
              fhe.Ciphertext(out.data[c * per:(c + 1) * per], LOGQ - K_RESCALE)) for c in range(nchunk)]
    in_free = [None] * nchunk   # compute of the previous step has read sub-batch c's inputs
    out_free = [None] * nchunk  # the previous step's download of sub-batch c's result is done

    def e2e_step():
        landed = []
        for c, (a_c, b_c, _) in enumerate(parts):
            with torch.cuda.stream(up):
                if in_free[c] is not None:
                    up.wait_event(in_free[c])
                a_c.data.copy_(A_h[c * per:(c + 1) * per], non_blocking=True)
                b_c.data.copy_(B_h[c * per:(c + 1) * per], non_blocking=True)
                landed.append(up.record_event())
        for c, (a_c, b_c, o_c) in enumerate(parts):
            with torch.cuda.stream(comp):
                comp.wait_event(landed[c])
                if out_free[c] is not None:
                    comp.wait_event(out_free[c])
                fhe.fhe_mult_relin_rescale(ctx, a_c, b_c, K_RESCALE, o_c)
                done = comp.record_event()
                in_free[c] = done
            with torch.cuda.stream(down):
                down.wait_event(done)
                out_h[c * per:(c + 1) * per].copy_(o_c.data, non_blocking=True)
                out_free[c] = down.record_event()

    def e2e_run(nsteps):
        """nsteps back-to-back steps; a step's uploads may start while the previous one computes."""
        main = torch.cuda.current_stream()
        for st in (up, comp, down):
            st.wait_stream(main)
        for _ in range(nsteps):
            e2e_step()
        for st in (up, comp, down):
            main.wait_stream(st)

    e2e_run(2)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    e2e_run(args.e2e_steps)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = f0.elapsed_time(f1)
    ms_e2e = max_over_ranks(ms_e2e, dist, "cuda")
    e2e_value = job_throughput(world, cnum, args.e2e_steps, ms_e2e)
    h2d = A_h.numel() * 4 + B_h.numel() * 4
    d2h = out_h.numel() * 4

    # latency of a single pair (cnum = 1)
    lat = []
    a1 = fhe.Ciphertext(A.data[:1].clone(), LOGQ)
    b1 = fhe.Ciphertext(B.data[:1].clone(), LOGQ)
    o1 = ctx.empty_ct(1, LOGQ - K_RESCALE)
    for i in range(args.latency_iters + 3):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        fhe.fhe_mult_relin_rescale(ctx, a1, b1, K_RESCALE, o1)
        s1.record(stream)
        s1.synchronize()
        if i >= 3:
            lat.append(s0.elapsed_time(s1))
    lat.sort()

    work = step_work(fhe, cnum, args.crt)
    times = {k: v[1] for k, v in prof.items()}
    dominant = max((k for k in times if k in work), key=lambda k: times[k])
    total_work = work[dominant] * args.steps
    achieved = total_work / (times[dominant] / 1e3) / 1e12  # Tslot/s or TFLOP/s
    nlaunch_dom = prof[dominant][0]
    traffic = read_traffic(dominant)
    if dominant in TENSOR_CLASSES.get(args.crt, ()):
        peaks = measured_peaks()
        peak = peaks.get("bf16_tflops_sustained") or 1700.0
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "peak_basis": ("measured dense bf16 (= fp16 nominal rate), sustained, MEASURED_PEAKS.json"
                               if peaks.get("bf16_tflops_sustained") else "fallback sustained bf16 1.7 PFLOP/s")}
    else:
        peak = SM_COUNT * IMAD_SLOTS_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "Tslot/s",
                "peak_basis": f"{SM_COUNT} SMs x {IMAD_SLOTS_PER_CLK} IMAD-pipe slots/clk x {SM_MAX_MHZ} MHz"}

    result = {
        "metric": METRIC, "value": value, "unit": "ct/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded encryptions of encoded-size plaintexts)",
        "config": {"workload": WORKLOAD, "cnum": cnum, "logN": LOGN, "logQ": LOGQ, "logP": LOGP, "crt": args.crt, "ntt": args.ntt,
                   "log_scale": K_RESCALE, "primes": work["primes"],
                   "l2": f"inputs larger than L2: {2 * A.data.numel() * 4 / 1e9:.2f} GB of ciphertexts per step"},
        "latency": {"cnum": 1, "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                    "iters": len(lat)},
        "e2e": {"value": e2e_value, "unit": "ct/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": args.e2e_steps, "sub_batches": nchunk,
                "streams": "upload, compute, download"},
        "gpu_launches": launches,
        "roofline": {"bound": roof["bound"], "kernel": dominant, "achieved": achieved, "peak": peak,
                     "unit": roof["unit"], "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": roof["peak_basis"], "launches": nlaunch_dom},
        "kernels": {k: class_roofline(k, n, t, work, args, sum(times.values())) for k, (n, t) in prof.items()},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, wall, per = oracle_throughput(1, 0, 1)
        result["cpu_baseline"] = {"value": v, "unit": "ct/s", "cores": 1, "kind": "oracle",
                                  "sample": "one ciphertext pair HMult+relin+rescale at the full workload size "
                                            f"({wall:.1f} s on one host core)"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def run_batched(args):
    """512 CKKS pairs, N in {2^13..2^16}, logQ uniform in [200, 1200], keys per N with logP = 1200:
    one CUDA-graph launch of the autotuned plan vs per-op launches, identical results."""
    import numpy as np
    import torch

    import fhe_synth as fs
    import paper_2607_05920_gb300 as fhe
    from paper_2607_05920_gb300 import batch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    g = fs.rng(4040)
    ctxs = {}
    for logN in (13, 14, 15, 16):
        N = 1 << logN
        c = fhe.Context(logN, 1200, 1200)
        c.keygen_inject(fs.ternary(g, (), N), fs.uniform_limbs(g, (), N, 1200), fs.gaussian(g, (), N),
                 fs.uniform_limbs(g, (), N, 2400), fs.gaussian(g, (), N))
        ctxs[logN] = c
    items = []
    for _ in range(args.cnum if args.cnum != 64 else 512):
        logN = int(g.choice([13, 14, 15, 16]))
        logQ = int(g.integers(200, 1201))
        N = 1 << logN
        mk = lambda: fhe.Ciphertext(torch.from_numpy(
            fs.uniform_limbs(g, (1, 2), N, logQ).view(np.int32).copy()).cuda(), logQ)
        items.append(batch.Item(logN, logQ, mk(), mk()))
    runner = batch.BatchRunner(ctxs, K_RESCALE)
    tuner = batch.Autotuner()
    tuned = tuner.tune(runner, items, reps=1)
    plan = runner.plan(items, tuned["schedule"])
    runner.pack(plan, items)
    form_ms = tuner.tune_forms(runner, plan, reps=2)
    branch_ms = tuner.tune_branches(runner, plan, reps=3)
    table_ms = tuner.tune_table(runner, plan, reps=2)
    runner.capture(plan)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        runner.graph.replay()
        runner.per_op(items)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        runner.graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / args.steps
    e0.record(stream)
    for _ in range(args.steps):
        ref = runner.per_op(items)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_per_op = e0.elapsed_time(e1) / args.steps
    runner.per_level(items)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        lev = runner.per_level(items)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_per_level = e0.elapsed_time(e1) / args.steps
    got = runner.outputs(plan, items)
    identical = all(torch.equal(got[i], ref[i].data[0]) and torch.equal(got[i], lev[i]) for i in range(len(items)))
    # per group: 2 lifts, 2 reconstructions, 1 signed lift and the 6 transform launches of its two ring
    # products (about 16 kernels with the limb work); the work-table call shares the 6 transform launches
    launches_graph = sum(16 for _ in plan.groups) if runner.table is None else 10 * len(plan.groups) + 6
    line = {
        "metric": "uneven-batch HMult+relin+rescale pairs/s (N 2^13..2^16, logQ 200..1200)",
        "value": len(items) / (ms_graph / 1e3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "dtype": "u32",
        "data": "synthetic (uniform ciphertexts, seeded)",
        "config": {"workload": "512 CKKS pairs, N uniform in {2^13..2^16}, logQ uniform in [200,1200], logP 1200, "
                               "scale 2^40, one CUDA-graph launch", "items": len(items),
                   "schedule": {str(k): v for k, v in tuned["schedule"].items()}, "groups": len(plan.groups)},
        "per_op": {"value": len(items) / (ms_per_op / 1e3), "ms_per_step": ms_per_op, "launches": 15 * len(items)},
        "per_level": {"value": len(items) / (ms_per_level / 1e3), "ms_per_step": ms_per_level,
                      "how": "one fhe_mult_relin_rescale per (ring, exact level), pairs of a level stacked"},
        "speedup_vs_per_op": ms_per_op / ms_graph, "speedup_vs_per_level": ms_per_level / ms_graph,
        "identical_results": bool(identical),
        "group_forms": [[g.logN, g.L_pad, len(g.idx), list(g.forms)] for g in plan.groups],
        "form_timings_ms": form_ms,
        "ring_branches": bool(runner.branches), "branch_timings_ms": branch_ms,
        "work_table": list(runner.table) if runner.table else None, "work_table_per_ring": runner.table_per_ring,
        "table_timings_ms": table_ms,
        "graph_kernels_approx": launches_graph,
        "autotune_ms": {str(k): v for k, v in tuned["timings_ms"].items()},
    }
    print(json.dumps(line), flush=True)
    for c in ctxs.values():
        c.close()


def run_serving(args):
    """Poisson arrivals of mult / rotate / degree-7 requests at N=2^16, logQ 1550 - 40k (k = 0..10)."""
    import numpy as np
    import torch

    import fhe_synth as fs
    import paper_2607_05920_gb300 as fhe
    from paper_2607_05920_gb300 import serve

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    logN, top = 16, 1550
    N = 1 << logN
    g = fs.rng(5050)
    ctx = fhe.Context(logN, top, top)
    ctx.keygen_inject(fs.ternary(g, (), N), fs.uniform_limbs(g, (), N, top), fs.gaussian(g, (), N),
               fs.uniform_limbs(g, (), N, 2 * top), fs.gaussian(g, (), N))
    steps = [1 << j for j in range(15)]
    for st in steps:
        ctx.keygen_rotation(st, fs.uniform_limbs(g, (), N, 2 * top), fs.gaussian(g, (), N))
    levels = [top - 40 * k for k in range(11)]
    pool_size = 8
    pool = {lq: fhe.Ciphertext(torch.from_numpy(
        fs.uniform_limbs(g, (pool_size, 2), N, lq).view(np.int32).copy()).cuda(), lq) for lq in levels}
    keep = lambda r: r.rid % 16 == 0  # noqa: E731  (results kept for the identity check: a sample)

    def drop(r):
        if not keep(r):
            r.result = None

    srv = serve.Server(ctx, pool, k=K_RESCALE, budget_bytes=80 << 30, max_batch=64, streams=2)
    srv.run(serve.make_requests(fs.rng(1), 200.0, 0.2, levels, pool_size, steps), on_done=drop)
    serve.run_per_op(ctx, pool, serve.make_requests(fs.rng(1), 200.0, 0.2, levels, pool_size, steps), K_RESCALE,
                     on_done=drop)
    reqs = serve.make_requests(g, args.rate, args.duration, levels, pool_size, steps)
    served, per = copy.deepcopy(reqs), copy.deepcopy(reqs)
    stats = srv.run(served, on_done=drop)
    pstats = serve.run_per_op(ctx, pool, per, K_RESCALE, on_done=drop)
    identical = all(torch.equal(a.result, b.result) for a, b in zip(served, per) if keep(a))
    checked = sum(1 for a in served if keep(a))
    del served, per
    low_reqs = serve.make_requests(fs.rng(7), 50.0, 1.0, levels, pool_size, steps)
    low = srv.run(copy.deepcopy(low_reqs), on_done=drop)
    plow = serve.run_per_op(ctx, pool, copy.deepcopy(low_reqs), K_RESCALE, on_done=drop)
    line = {
        "metric": "served homomorphic requests/s (N=2^16, logQ 1150..1550, mult/rotate/poly7 = 50/30/20%)",
        "value": stats["ops_per_s"], "unit": "req/s", "n_gpus": 1, "higher_is_better": True, "dtype": "u32",
        "data": "synthetic (Poisson arrivals, uniform ciphertexts, seeded)",
        "config": {"workload": "continuous batching, keys resident, admission by HBM footprint",
                   "offered_rate_hz": args.rate, "arrival_window_s": args.duration, "streams": 2, "max_batch": 64,
                   "budget_gb": 80, "levels": levels},
        "latency_ms": {"p50": stats["p50_ms"], "p99": stats["p99_ms"]}, "completed": stats["completed"],
        "offered": stats["offered"], "wall_s": stats["wall_s"], "by_op": stats["by_op"],
        "saturated": stats["ops_per_s"] < 0.95 * args.rate,
        "per_op": {"ops_per_s": pstats["ops_per_s"], "p50_ms": pstats["p50_ms"], "p99_ms": pstats["p99_ms"],
                   "wall_s": pstats["wall_s"], "how": "each request alone through the plain calls as it arrives, "
                                                     "one stream, at most 256 in flight"},
        "identical_results": bool(identical), "identity_checked_requests": checked,
        "low_load": {"offered_rate_hz": 50.0, "served": {k: low[k] for k in ("ops_per_s", "p50_ms", "p99_ms")},
                     "per_op": {k: plow[k] for k in ("ops_per_s", "p50_ms", "p99_ms")}},
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_rotations(args):
    """The sparse-secret workload: N=2^15, logQ=logP=880, Hamming-weight-64 secret, scale 2^40; a batch of
    64 pairs multiplied, relinearised and rescaled, then every product rotated by the 15 power-of-two
    steps 2^0..2^14 (hoisted: one lift and forward transform per batch, 15 transform-domain gathers)."""
    import numpy as np
    import torch

    import paper_2607_05920_gb300 as fhe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    logN, logQ, k, cnum = 15, 880, K_RESCALE, args.cnum
    N = 1 << logN
    steps = [1 << j for j in range(15)]
    ctx = fhe.Context(logN, logQ, logQ, hamming_weight=64)
    ctx.keygen(0xC2, rot_steps=steps)
    g = np.random.Generator(np.random.PCG64(215))
    L = fhe.limbs(logQ)

    def pt_batch():
        # encoded-message-sized signed coefficients as two's-complement limbs mod 2^logQ
        m = g.integers(-(1 << 41) + 1, 1 << 41, size=(cnum, N), dtype=np.int64)
        pt = np.zeros((cnum, L, N), dtype=np.uint32)
        mu = m.astype(np.uint64)
        pt[:, 0] = (mu & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        pt[:, 1] = (mu >> np.uint64(32)).astype(np.uint32)
        for l in range(2, L):
            pt[:, l] = np.where(m < 0, np.uint32(0xFFFFFFFF), 0)
        top = logQ - 32 * (L - 1)
        pt[:, L - 1] &= np.uint32((1 << top) - 1)
        return torch.from_numpy(pt.view(np.int32)).cuda()

    A = ctx.encrypt(pt_batch(), 1, log_scale=40)
    B = ctx.encrypt(pt_batch(), 2, log_scale=40)
    prod = ctx.empty_ct(cnum, logQ - k)
    outs = [ctx.empty_ct(cnum, logQ - k) for _ in steps]
    ctx.workspace(fhe.FHE_OP_MULT, logQ, cnum)
    ctx.workspace(fhe.FHE_OP_ROTATE, logQ - k, cnum)

    def step_hoisted():
        fhe.fhe_mult_relin_rescale(ctx, A, B, k, prod)
        fhe.fhe_rotate_hoisted(ctx, prod, steps, outs)

    def step_separate():
        fhe.fhe_mult_relin_rescale(ctx, A, B, k, prod)
        for s_, o in zip(steps, outs):
            fhe.fhe_rotate(ctx, prod, s_, o)

    def timed(fn, n):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    clocks = ClockSampler(0)
    clocks.start()
    ms_h = timed(step_hoisted, args.steps)
    clk = clocks.stop()
    ref = [o.data.clone() for o in outs]
    ms_s = timed(step_separate, args.steps)
    identical = all(torch.equal(r, o.data) for r, o in zip(ref, outs))
    # the multiplication alone, to split the step
    ms_m = timed(lambda: fhe.fhe_mult_relin_rescale(ctx, A, B, k, prod), args.steps)
    line = {
        "metric": "ciphertext pairs/s through HMult+relin+rescale and 15 power-of-two rotations (N=2^15, logQ=880)",
        "value": cnum / (ms_h / 1e3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_h, "higher_is_better": True, "dtype": "u32",
        "data": "synthetic (seeded keys and encryptions of encoded-size plaintexts)",
        "config": {"workload": "CKKS N=2^15 logQ=logP=880, Hamming-weight-64 secret, scale 2^40, 64 pairs, "
                               "rotations by 2^0..2^14", "cnum": cnum},
        "rotations_per_s": {"hoisted": 15 * cnum / ((ms_h - ms_m) / 1e3),
                            "separate_calls": 15 * cnum / ((ms_s - ms_m) / 1e3)},
        "ms": {"step_hoisted": ms_h, "step_separate": ms_s, "mult_only": ms_m},
        "hoisting_speedup_on_rotations": (ms_s - ms_m) / (ms_h - ms_m),
        "identical_results": bool(identical), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_bgv(args):
    """BGV at N=2^14, t=65537, chain Q_l = q0 r^l (q0 ~ 2^54, r ~ 2^48, 8 levels, logQ=438, P = 2^438): a batch of
    128 ciphertexts squared 8 times with relinearisation and a modulus switch after each; the decryptions are
    checked against m^(2^8) mod (X^N + 1, t) computed on the GPU by the same scheme's plaintext rule."""
    import numpy as np
    import torch

    import paper_2607_05920_gb300 as fhe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t, levels, logN, cnum = 65537, 8, 14, 128
    # q0, r: the largest odd values = 1 mod t below 2^54 and 2^48 (as the tests choose them)
    def pick(bits):
        k = ((1 << bits) - 1) // t
        if (1 + t * k) % 2 == 0:
            k -= 1
        return 1 + t * k

    q0, r = pick(54), pick(48)
    logQ = (q0 * r ** levels).bit_length()
    ctx = fhe.Context(logN, logQ, logQ, scheme=fhe.FHE_SCHEME_BGV, t=t, bgv_q0=q0, bgv_r=r, bgv_levels=levels)
    ctx.keygen(0xB6)
    N = 1 << logN
    g = np.random.Generator(np.random.PCG64(303))
    slots = torch.from_numpy(g.integers(0, t, size=(cnum, N), dtype=np.int64).astype(np.int32)).cuda()
    ct0 = ctx.encrypt(fhe.fhe_bgv_encode(ctx, slots, logQ), 5)

    def chain():
        ct = ct0
        for _ in range(levels):
            ct = ctx.mod_switch(ctx.mult_relin(ct, ct))
        return ct

    for _ in range(args.warmup):
        out = chain()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    e0.record()
    for _ in range(args.steps):
        out = chain()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # slot-wise: x^(2^8) mod t in every slot
    want = slots.to(torch.int64)
    for _ in range(levels):
        want = want * want % t
    got = fhe.fhe_bgv_decode(ctx, ctx.decrypt(out)).to(torch.int64)
    line = {
        "metric": "BGV ciphertexts/s through a depth-8 squaring chain with relinearisation and modulus switching "
                  "(N=2^14, logQ=438, t=65537)",
        "value": cnum / (ms / 1e3), "unit": "ct/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "u32",
        "data": "synthetic (seeded keys and encryptions of slot-encoded uniform plaintexts mod t)",
        "config": {"workload": "BGV N=2^14, chain q0 r^8 (logQ 438), P=2^438, t=65537, 128 ciphertexts, "
                               "8 squarings", "cnum": cnum},
        "homomorphic_mults_per_s": levels * cnum / (ms / 1e3),
        "decryptions_exact": bool(torch.equal(got, want)), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.workload == "serving" and args.impl != "reference":
        run_serving(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "rotations":
        run_rotations(args)
    elif args.workload == "bgv":
        run_bgv(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
