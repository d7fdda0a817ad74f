#!/usr/bin/env python
"""Benchmark of the Ozaki-II multiple-precision GEMM on GB300.

Workload: one M = N = K = 1024 product at p = 256 bits (256 random
significand bits with the top bit set, random sign, exponents i.i.d. uniform
in [-32, 32]; seeded synthetic data).  A step is one whole product: exponent
scan, integerization + residues, the grouped plane GEMM with fused
mod-reduce, CRT and rounding.  `value` is whole-job 2MNK per second with the
inputs resident in HBM; `e2e` times the same products through the C ABI with
host buffers: every step copies A and B from pinned host memory and C back,
inside the timed region, double-buffered so that the copies of neighbouring
steps overlap the product.  L2 is flushed (a 512 MiB write) between the
device-resident steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica of
the workload (the path needs no exchange); the time is the max over ranks.
`--impl reference` times the CPU oracle (the slow, exact stage-by-stage
restatement of the method) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p-bit GEMM 2MNK/s at p=53–2048; INT8 TC util; batched vs plain speedup"
UNIT = "2MNK/s"
WORK = {"workload": "gemm_1024_p256", "M": 1024, "N": 1024, "K": 1024, "p": 256,
        "exp_range": [-32, 32], "seed": 1001}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
CPU_BLOCK = 32          # oracle sample: 32 x 32 output blocks of the workload


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dev) -> float:
    """The largest of every rank's x (the slowest replica sets the job time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, work_per_rank: float, ms: float) -> float:
    """Whole-job rate: every rank runs its own replica of the workload, so the
    job does world x work in the max-over-ranks time."""
    return world * work_per_rank / (ms / 1e3)


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------

def _oracle_block(args):
    i0, j0 = args
    import synth
    from oracle import ozaki2_oracle as o
    A, B = synth.gemm_1024_p256(WORK["seed"])
    rows = slice(i0, i0 + CPU_BLOCK)
    cols = slice(j0, j0 + CPU_BLOCK)
    As = {"p": A["p"], "limbs": A["limbs"][:, rows, :].copy(), "exp": A["exp"][rows, :].copy(),
          "sign": A["sign"][rows, :].copy()}
    Bs = {"p": B["p"], "limbs": B["limbs"][:, :, cols].copy(), "exp": B["exp"][:, cols].copy(),
          "sign": B["sign"][:, cols].copy()}
    t = time.perf_counter()
    o.ozaki2_full(As, Bs, WORK["p"])
    return time.perf_counter() - t


def cpu_oracle_rate(rounds: int = 2):
    """Time the CPU oracle (stage-by-stage method, exact integers) on a bounded
    sample: `cores * rounds` blocks of 32 x 32 outputs (full K) of the
    workload, one spawn-pool process per host core."""
    cores = os.cpu_count() or 1
    nblk = cores * rounds
    offs = [((b * 97) % (WORK["M"] // CPU_BLOCK) * CPU_BLOCK, (b * 61) % (WORK["N"] // CPU_BLOCK) * CPU_BLOCK)
            for b in range(nblk)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_block, offs, chunksize=1)
    wall = time.perf_counter() - t0
    work = nblk * 2 * CPU_BLOCK * CPU_BLOCK * WORK["K"]
    sample = (f"oracle ozaki2_full on {nblk} blocks of {CPU_BLOCK}x{CPU_BLOCK} outputs (full K=1024) of "
              f"the 1024^3 p=256 workload, spawn pool of {cores} processes, wall {wall:.1f} s "
              f"incl. input regeneration")
    return work / wall, cores, sample


# ---------------------------------------------------------------------------
# roofline of each stage
# ---------------------------------------------------------------------------

# Integer-pipe rates per SM per clock used as the ALU peaks: 64 lanes of
# 32-bit integer multiply-add per SM per clock (the FMA-heavy pipe: 4 SM
# sub-partitions x 16 lanes); a 32 x 32 -> 64-bit multiply-add (IMAD.WIDE)
# takes two passes, and a 4-way byte dot product (dp4a) one pass for four
# multiply-adds.  Times 152 SMs and the maximum SM clock.
SMS = 152
IMAD_WIDE_PER_SM_CLK = 32
DP4A_MACS_PER_SM_CLK = 64 * 4

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of the committed kernels on the same workload; the source
# summaries are under profiles/.  A kernel changed since its capture has None.
NCU_TRAFFIC = {
    "gemm_1024_p256": {"residues": 443.90144e6, "gemm": 564.279552e6, "crt_sums": 223.868672e6,
                       "crt_finish": 123.980288e6},
}


def stage_rooflines(info, M, N, K, p, stages, workload):
    """Achieved vs peak for each stage's kernel, from its algorithmic work.

    residues: byte multiply-adds sum_b beta_b (2^(8b) mod m) over the
      ceil((t+1)/8) bytes of each integerized entry, one per modulus for the
      L1 one-limb moduli and two (the low and high table byte) for the L2
      two-limb moduli: (M+N) K ceil((t+1)/8) (L1 + 2 L2), against the dp4a
      multiply-add rate.
    gemm: 2 M N K G flops of the G plane products, against the measured bf16
      tensor peak (the integer planes are exact bf16 operands).
    crt (CUDA-core CRT): the 32 x 32 -> 64-bit multiply-adds of
      sum_l v_l M_l, L per output and digit of M_l: M N L ceil(bits(P)/32),
      against the IMAD.WIDE rate.
    crt_sums (tensor-core CRT): the exact bf16 products of the column sums
      Y = V B, 2 M N (2L) np flops with np 7-bit pieces of P, against the
      bf16 tensor peak.
    crt_finish (after the sums): the bytes it moves, the group words it reads
      (D + 2 ceil(D/7) per output), the 4-byte quotient estimate and the
      output (8 nl + 5 bytes), against HBM.
    scan: the bytes of the two exponent vectors' inputs, against HBM.

    Every stage also carries ``hbm``: its algorithmic bytes (what it must read
    and write once) over its time, against the measured HBM copy rate, whatever
    its own bound: residues read the inputs (8 nl + 5 bytes per entry) and
    write the G bf16 planes; the GEMM reads both plane stacks and writes the L
    16-bit values v_l; the CRT reads v_l and writes C (8 nl + 5 bytes per
    output), the tensor-core sums writing the 9-word group sums and the 4-byte
    estimate in between.
    """
    peaks, src = load_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    L, L1, G, t = info["L"], info["L1"], info["G"], info["t"]
    L2 = L - L1
    md = info["crt_digits"] - 2
    traffic = NCU_TRAFFIC.get(workload, {})
    out = {}

    def alu(name, kernel, ops, rate, what):
        ach = ops / (stages[name] / 1e3) / 1e12
        out[name] = {"kernel": kernel, "bound": "alu", "achieved": round(ach, 2),
                     "peak": round(rate / 1e12, 2), "unit": f"T{what}/s", "frac": round(ach * 1e12 / rate, 4),
                     "peak_source": f"{SMS} SMs x {rate / SMS / clk:.0f} {what}/SM/clk x "
                                    f"{clk / 1e6:.0f} MHz (derived)",
                     "traffic": traffic.get(name)}

    res_macs = (M + N) * K * math.ceil((t + 1) / 8) * (L1 + 2 * L2)
    alu("residues", "k_residue (integerize + byte-table residues + plane writes)", res_macs,
        SMS * DP4A_MACS_PER_SM_CLK * clk, "byteMAC")
    if "crt" in stages:
        alu("crt", "k_crt1 / k_crt (direct CRT sum + quotient correction + rounding)", M * N * L * md,
            SMS * IMAD_WIDE_PER_SM_CLK * clk, "imad64")
    if "crt_sums" in stages:
        np_ = info["crt_pieces"]
        fl = 2.0 * M * N * (2 * L) * np_
        ach = fl / (stages["crt_sums"] / 1e3) / 1e12
        pk = float(peaks["bf16_tflops"])
        out["crt_sums"] = {"kernel": "k_crt_mm (CRT column sums as an exact bf16 GEMM + group carries)",
                           "bound": "tensor", "achieved": round(ach, 1), "peak": pk, "unit": "TFLOP/s",
                           "frac": round(ach / pk, 4), "peak_source": f"bf16_tflops burst, {src}",
                           "traffic": traffic.get("crt_sums")}
        D = info["crt_digits"]
        nl = -(-p // 64)
        fb = M * N * (4 * (D + 2 * -(-D // 7)) + 4 + 8 * nl + 5)
        ach = fb / (stages["crt_finish"] / 1e3) / 1e9
        pk = float(peaks["hbm_gbs"])
        out["crt_finish"] = {"kernel": "k_crt_fin_long (CRT finish from the group sums + rounding)",
                             "bound": "hbm", "achieved": round(ach, 1), "peak": pk, "unit": "GB/s",
                             "frac": round(ach / pk, 4), "peak_source": f"hbm_gbs, {src}",
                             "traffic": traffic.get("crt_finish")}
    flops = 2.0 * M * N * K * G
    ach = flops / (stages["gemm"] / 1e3) / 1e12
    pk = float(peaks["bf16_tflops"])
    out["gemm"] = {"kernel": "k_gemm_tc (plane GEMMs + fused mod-reduce)", "bound": "tensor",
                   "achieved": round(ach, 1), "peak": pk, "unit": "TFLOP/s", "frac": round(ach / pk, 4),
                   "peak_source": f"bf16_tflops burst, {src}", "traffic": traffic.get("gemm")}
    scan_bytes = (M * K + K * N) * (8 + 4)      # top limb + exponent of every entry
    ach = scan_bytes / (stages["scan"] / 1e3) / 1e9
    pk = float(peaks["hbm_gbs"])
    out["scan"] = {"kernel": "k_scan (shared exponents)", "bound": "hbm", "achieved": round(ach, 1),
                   "peak": pk, "unit": "GB/s", "frac": round(ach / pk, 4),
                   "peak_source": f"hbm_gbs, {src}", "traffic": traffic.get("scan")}
    nl = -(-p // 64)
    Kp = -(-K // 8) * 8
    io_in = (M * K + K * N) * (8 * nl + 5)
    c_out = M * N * (8 * nl + 5)
    v_bytes = L * M * N * 2
    nbytes = {"scan": (M * K + K * N) * (8 + 4),
              "residues": io_in + G * (M + N) * Kp * 2,
              "gemm": G * (M + N) * Kp * 2 + v_bytes,
              "crt": v_bytes + c_out}
    if "crt_sums" in stages:
        ngrp = -(-(info["crt_pieces"] + 5) // 32)
        D = info["crt_digits"]
        nbytes["crt_sums"] = v_bytes + M * N * (ngrp * 9 * 4 + 4)
        nbytes["crt_finish"] = M * N * (4 * (D + 2 * -(-D // 7)) + 4) + c_out
    hpk = float(peaks["hbm_gbs"])
    for name, ms in stages.items():
        if name in out and name in nbytes:
            gbs = nbytes[name] / (ms / 1e3) / 1e9
            out[name]["hbm"] = {"bytes": nbytes[name], "achieved": round(gbs, 1), "peak": hpk, "unit": "GB/s",
                                "frac": round(gbs / hpk, 4)}
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as ozk

    world, rank, local = dist_info()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    # the CPU baseline's spawn pool runs before the first CUDA call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(args.cpu_rounds)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    M, N, K, p = WORK["M"], WORK["N"], WORK["K"], WORK["p"]
    A, B = synth.gemm_1024_p256(WORK["seed"])
    dA, dB = ozk.MPMatrix.from_host(A, dev), ozk.MPMatrix.from_host(B, dev)
    dC = ozk.MPMatrix.empty(M, N, p, dev)
    plan = ozk.Plan((M, N, K, p), timing=1)
    ws = plan.workspace(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        plan.execute(dA, dB, dC, ws)
    plan.check()
    torch.cuda.synchronize()

    # ---- device-resident timing
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = []
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    clk = ClockSampler(f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-")
                       else (str(uuid) if uuid is not None else local))
    clk.start()
    barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(s & 0xff)
        starts[s].record(stream)
        plan.execute(dA, dB, dC, ws)
        ends[s].record(stream)
        stage.append({**plan.timings(), **plan.crt_split()})
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    plan.check()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dev)
    work = 2.0 * M * N * K
    value = replica_value(world, work, ms)

    # ---- end to end through the C ABI with host buffers
    hA = {k: torch.from_numpy(np.ascontiguousarray(A[k]).view(np.int64) if k == "limbs" else
                              np.ascontiguousarray(A[k])).pin_memory() for k in ("limbs", "exp", "sign")}
    hB = {k: torch.from_numpy(np.ascontiguousarray(B[k]).view(np.int64) if k == "limbs" else
                              np.ascontiguousarray(B[k])).pin_memory() for k in ("limbs", "exp", "sign")}
    hC = {"limbs": torch.empty(dC.limbs.shape, dtype=torch.int64).pin_memory(),
          "exp": torch.empty(dC.exp.shape, dtype=torch.int32).pin_memory(),
          "sign": torch.empty(dC.sign.shape, dtype=torch.int8).pin_memory()}
    h2d = sum(v.numel() * v.element_size() for v in list(hA.values()) + list(hB.values()))
    d2h = sum(v.numel() * v.element_size() for v in hC.values())
    # double-buffered: the host->device copies of step s + 1 (stream s_in) and the
    # device->host copy of step s - 1 (stream s_out) overlap the product of step s
    # (the launch stream); every step's copies are inside the timed region, which
    # runs from before the first input copy to after the last output copy
    bufA = [dA, ozk.MPMatrix.from_host(A, dev)]
    bufB = [dB, ozk.MPMatrix.from_host(B, dev)]
    bufC = [dC, ozk.MPMatrix.empty(M, N, p, dev)]
    hCs = [hC, {k: torch.empty_like(v).pin_memory() for k, v in hC.items()}]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def copy_in(sidx):
        b = sidx & 1
        with torch.cuda.stream(s_in):
            if sidx >= 2:
                s_in.wait_event(ev_done[b])          # the product of step sidx - 2 has read buffer b
            for dst, src in ((bufA[b], hA), (bufB[b], hB)):
                dst.limbs.copy_(src["limbs"], non_blocking=True)
                dst.exp.copy_(src["exp"], non_blocking=True)
                dst.sign.copy_(src["sign"], non_blocking=True)
            ev_in[b].record(s_in)

    def copy_out(sidx):
        b = sidx & 1
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[b])
            for k in ("limbs", "exp", "sign"):
                hCs[b][k].copy_(getattr(bufC[b], k), non_blocking=True)
            ev_out[b].record(s_out)

    barrier()
    torch.cuda.synchronize()
    t0.record(s_in)
    copy_in(0)
    for st in range(args.steps):
        b = st & 1
        if st + 1 < args.steps:
            copy_in(st + 1)
        stream.wait_event(ev_in[b])
        if st >= 2:
            stream.wait_event(ev_out[b])             # the output copy of step st - 2 has read C[b]
        plan.execute(bufA[b], bufB[b], bufC[b], ws)
        ev_done[b].record(stream)
        copy_out(st)
    s_in.wait_stream(s_out)
    t1.record(s_in)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, dev)

    # ---- roofline of the dominant kernel (library stage events on the launch stream)
    med = {k: statistics.median(s_[k] for s_ in stage) for k in stage[0]}
    info = dict(plan.info)
    if info["crt_mode"] == 2:        # two kernels: the sums on the tensor cores, then the finish
        stages = {k: med[k] for k in ("scan", "residues", "gemm", "crt_sums", "crt_finish")}
        Pm = 1
        for m in plan.moduli():
            Pm *= m
        info["crt_pieces"] = (Pm.bit_length() + 6) // 7 + 1
    else:
        stages = {k: med[k] for k in ("scan", "residues", "gemm", "crt")}
    kernels = stage_rooflines(info, M, N, K, p, stages, WORK["workload"])
    dom = max(stages, key=stages.get)
    roof = dict(kernels[dom])
    roof["stage_ms"] = {k: round(v, 4) for k, v in stages.items()}
    gemm_tflops = 2.0 * M * N * K * info["G"] / (stages["gemm"] / 1e3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16-int (exact integer planes on tcgen05 kind::f16)",
        "data": "synthetic", "impl": "ours",
        "config": {"workload": WORK["workload"], "M": M, "N": N, "K": K, "p": p,
                   "exp_range": WORK["exp_range"], "t": info["t"], "moduli": info["L"], "gemms": info["G"],
                   "parallelism": f"replicas{world}", "l2": "flushed (512 MiB write between steps)"},
        "e2e": {"value": replica_value(world, work, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "copies": "pinned host buffers, every step, double-buffered on two copy streams"},
        "roofline": roof,
        "kernels": {k: v for k, v in kernels.items() if k != dom},
        "plane_gemm_tflops": round(gemm_tflops, 1),
        "gpu_launches": plan.launches() * args.steps,
        "clocks": clocks,
    }
    if cpu is not None:
        rate, cores, sample = cpu
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_other(args):
    """Measurements of the other workloads (one GPU): batched, autograd, large."""
    import numpy as np
    import torch

    import synth
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as ozk
    from paper_2609_27831_gb300 import autograd as ag

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for s_ in range(steps):
            flush.fill_(s_ & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    out = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "data": "synthetic", "impl": "ours"}
    if args.workload == "batched64":
        probs = synth.batched_problems(64, 1002)
        shapes = [(M, N, K, p) for (M, N, K, p, _, _) in probs]
        trip = [(ozk.MPMatrix.from_host(A, dev), ozk.MPMatrix.from_host(B, dev), ozk.MPMatrix.empty(M, N, p, dev))
                for (M, N, K, p, A, B) in probs]
        work = sum(2.0 * M * N * K for (M, N, K, p) in shapes)
        plan_g = ozk.Plan(shapes)
        ws_g = plan_g.workspace(dev)
        s = torch.cuda.Stream(dev)
        with torch.cuda.stream(s):
            g = plan_g.graph(trip, ws_g, s)
        ms_graph = timed(lambda: g.launch(stream), args.steps, args.warmup)
        ms_grouped = timed(lambda: plan_g.execute_batched(trip, ws_g, stream), args.steps, args.warmup)
        del ws_g
        torch.cuda.empty_cache()
        plan_p = ozk.Plan(shapes, schedule=1)
        ws_p = plan_p.workspace(dev)
        ms_plain = timed(lambda: plan_p.execute_batched(trip, ws_p, stream), args.steps, args.warmup)
        plan_p.check()
        out.update({"value": work / (ms_graph / 1e3), "ms_per_step": ms_graph,
                    "config": {"workload": "batched64", "problems": 64, "M_N_K": "log-uniform [128, 2048]",
                               "p": [113, 256, 512], "gemms": sum(1 for _ in shapes)},
                    "batched": {"graph_ms": ms_graph, "grouped_ms": ms_grouped, "plain_ms": ms_plain,
                                "speedup_vs_plain": ms_plain / ms_graph,
                                "plain": "one GEMM launch per modulus per problem (other stages grouped)"}})
    elif args.workload == "dgemm4096_autograd":
        X, Y, G = synth.fp64_workload(4096, 1003)
        xa = torch.tensor(X, device=dev, requires_grad=True)
        ya = torch.tensor(Y, device=dev, requires_grad=True)
        gt = torch.tensor(G, device=dev)

        def step():
            xa.grad = None
            ya.grad = None
            ag.ozaki_matmul(xa, ya).backward(gt)
        ms = timed(step, args.steps, args.warmup)
        n = 4096
        out.update({"value": 3 * 2.0 * n ** 3 / (ms / 1e3), "ms_per_step": ms,
                    "config": {"workload": "dgemm4096_autograd", "M": n, "N": n, "K": n, "p": 53,
                               "step": "forward C = AB and backward dA, dB (3 products)"}})
    else:
        M, N, K, p, lo, hi = {"gemm_4096_p2048": (4096, 4096, 4096, 2048, -64, 64),
                              "gemm_8192_p53": (8192, 8192, 8192, 53, -8, 8),
                              "gemm_4096_p53": (4096, 4096, 4096, 53, -8, 8),
                              "gemm_2048_p512": (2048, 2048, 2048, 512, -8, 8)}[args.workload]
        A, B = synth.workload_single(M, N, K, p, lo, hi, 1004)
        dA, dB = ozk.MPMatrix.from_host(A, dev), ozk.MPMatrix.from_host(B, dev)
        del A, B
        dC = ozk.MPMatrix.empty(M, N, p, dev)
        plan = ozk.Plan((M, N, K, p), timing=1)
        ws = plan.workspace(dev)
        ms = timed(lambda: plan.execute(dA, dB, dC, ws), args.steps, args.warmup)
        plan.check()
        st = plan.timings()
        out.update({"value": 2.0 * M * N * K / (ms / 1e3), "ms_per_step": ms,
                    "config": {"workload": args.workload, "M": M, "N": N, "K": K, "p": p, "t": plan.info["t"],
                               "moduli": plan.info["L"], "gemms": plan.info["G"],
                               "workspace_gb": round(plan.workspace_bytes / 1e9, 2)},
                    "stage_ms": {k: round(v, 3) for k, v in st.items()},
                    "plane_gemm_tflops": round(2.0 * M * N * K * plan.info["G"] / (st["gemm"] / 1e3) / 1e12, 1)})
    print(json.dumps(out), flush=True)


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    for _ in range(args.warmup):
        _oracle_block((0, 0))
    rates = []
    for _ in range(args.steps):
        rate, cores, sample = cpu_oracle_rate(1)
        rates.append(rate)
    value = statistics.median(rates)
    ms = 2.0 * WORK["M"] * WORK["N"] * WORK["K"] / value * 1e3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "exact integers (Python)", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": WORK["workload"], "M": WORK["M"], "N": WORK["N"], "K": WORK["K"],
                   "p": WORK["p"], "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rounds", type=int, default=6)
    ap.add_argument("--workload", default="gemm_1024_p256",
                    choices=["gemm_1024_p256", "batched64", "dgemm4096_autograd", "gemm_4096_p2048",
                             "gemm_8192_p53", "gemm_4096_p53", "gemm_2048_p512"])
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "gemm_1024_p256":
        run_other(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
