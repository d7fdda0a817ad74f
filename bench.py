#!/usr/bin/env python
"""Benchmark of the Ozaki-II multiple-precision GEMM on GB300.

Default workload: the largest single-GPU configuration, one M = N = K = 4096
product at p = 2048 bits (2048 random significand bits with the top bit set,
random sign, exponents i.i.d. uniform in [-64, 64]; seeded synthetic data),
with the residue planes streamed through the workspace in groups of moduli.
A step is one whole product: exponent scan, integerization + residues, the
grouped plane GEMMs with fused mod-reduce, CRT and rounding.  `value` is
whole-job 2MNK per second with the inputs resident in HBM; `e2e` times the
same products through the C ABI with host buffers: every step copies A and B
from pinned host memory and C back, inside the timed region, double-buffered
so that the copies of neighbouring steps overlap the product.  L2 is flushed
(a 512 MiB write) between device-resident steps, outside the timed events.

The same JSON line carries a `sweep` over the rest of the metric: the
1024^3 p = 256 and 8192^3 p = 53 products, the 64-problem batch in one CUDA
graph against the plain one-launch-per-modulus form, the binary64 autograd
step at 4096^2, and the INT8 tensor-core peak of this GPU (the library's
mma.sync s8 probe and torch._int_mm) with the plane GEMMs' exact-integer
rate against it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--no-sweep] [--no-e2e] [--no-cpu-baseline]

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica of
the workload (the path needs no exchange); the time is the max over ranks.
`--impl reference` times the CPU oracle (the slow, exact stage-by-stage
restatement of the method) on the host cores instead, on sampled output
entries of the same workload.
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
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}

# single-product workloads: M, N, K, p, exponent range, seed
WORKLOADS = {
    "gemm_4096_p2048": (4096, 4096, 4096, 2048, (-64, 64), 1004),   # large, p = 2048
    "gemm_8192_p53": (8192, 8192, 8192, 53, (-8, 8), 1004),         # large, p = 53
    "gemm_1024_p256": (1024, 1024, 1024, 256, (-32, 32), 1001),     # one product, p = 256
    "gemm_256_p53": (256, 256, 256, 53, (-8, 8), 1000),             # small, p = 53
    "gemm_4096_p53": (4096, 4096, 4096, 53, (-8, 8), 1004),
    "gemm_2048_p512": (2048, 2048, 2048, 512, (-8, 8), 1004),
    "gemm_1024_p2048": (1024, 1024, 1024, 2048, (-64, 64), 1001),
    "gemm_1024_p53": (1024, 1024, 1024, 53, (-8, 8), 1001),
}
DEFAULT_WORKLOAD = "gemm_4096_p2048"
# a kernel timed inside a timed region longer than this runs under the power
# cap: its roofline uses the sustained bf16 peak, otherwise the burst peak
SUSTAINED_AFTER_S = 1.0


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

    def __init__(self, device_index):
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

def sample_entries(M: int, N: int, count: int, seed: int = 77):
    """Seeded sample of output entries (i, j) of an M x N product."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(int(rng.integers(M)), int(rng.integers(N))) for _ in range(count)]


def entry_tasks(A: dict, B: dict, pairs):
    """One oracle task per sampled entry: row i of A and column j of B only
    (the pool processes receive these slices, not the whole matrices)."""
    tasks = []
    for i, j in pairs:
        a = {"p": A["p"], "limbs": A["limbs"][:, i:i + 1, :].copy(), "exp": A["exp"][i:i + 1, :].copy(),
             "sign": A["sign"][i:i + 1, :].copy()}
        b = {"p": B["p"], "limbs": B["limbs"][:, :, j:j + 1].copy(), "exp": B["exp"][:, j:j + 1].copy(),
             "sign": B["sign"][:, j:j + 1].copy()}
        tasks.append((a, b))
    return tasks


def _oracle_entry(task):
    """The oracle's stage-by-stage method on one output entry (full K)."""
    from oracle import ozaki2_oracle as o
    a, b = task
    o.ozaki2_entries(a, b, a["p"], [(0, 0)])
    return 1


class OracleTimer:
    """Times the CPU oracle, as it stands, on sampled output entries of a
    workload: one spawn-pool process per host core, one entry per task."""

    def __init__(self, A: dict, B: dict, K: int, cores: int | None = None):
        self.cores = cores or os.cpu_count() or 1
        self.K = K
        M, N = A["exp"].shape[0], B["exp"].shape[1]
        self.pool_tasks = entry_tasks(A, B, sample_entries(M, N, 4 * self.cores))
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.done = 0

    def batch(self, n: int):
        """Run n entries (cycling through the sample); returns (entries, wall s)."""
        tasks = [self.pool_tasks[(self.done + q) % len(self.pool_tasks)] for q in range(n)]
        self.done += n
        t0 = time.perf_counter()
        self.pool.map(_oracle_entry, tasks, chunksize=1)
        return n, time.perf_counter() - t0

    def rate(self, min_s: float = 10.0, max_s: float = 30.0):
        """Batches of `cores` entries until at least min_s of wall time (and
        not more batches once max_s is passed): 2K per entry over the wall."""
        n_tot, wall = 0, 0.0
        while wall < min_s:
            n, w = self.batch(self.cores)
            n_tot += n
            wall += w
            if wall > max_s:
                break
        return n_tot * 2.0 * self.K / wall, n_tot, wall

    def close(self):
        self.pool.close()
        self.pool.join()


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

# DRAM traffic of each stage per execute (dram__bytes_read.sum +
# dram__bytes_write.sum over the stage's launches, averaged over the four
# executes of one ncu capture of the committed kernels on the same workload,
# one pass, the full size; the finish at 1024^3, p = 256 from its own
# capture of one launch after its last change); the source summaries are
# under profiles/.  A kernel changed since its capture is absent.
NCU_TRAFFIC = {
    "gemm_4096_p2048": {"scan": 403911680, "residues": 82033706496, "gemm": 121773933248,
                        "crt_sums": 20133005952, "crt_finish": 11299742848},
    "gemm_1024_p256": {"scan": 25205376, "residues": 440525568, "gemm": 562085952,
                       "crt_finish": 125142528},
}


def finish_kernel(crt_digits: int) -> str:
    """The finish kernel the library runs after the tensor-core CRT sums: the
    register finish up to 24 accumulator digits, the shared-memory one above."""
    return "k_crt_fin_short" if crt_digits <= 24 else "k_crt_fin_long"


def stage_rooflines(info, M, N, K, p, stages, workload, sustained: bool = False):
    """Achieved vs peak for each stage's kernel, from its algorithmic work.

    residues: byte multiply-adds sum_b beta_b (2^(8b) mod m) over the
      ceil((t+1)/8) bytes of each integerized entry, one per modulus for the
      L1 one-limb moduli and two (the low and high table byte) for the L2
      two-limb moduli: (M+N) K ceil((t+1)/8) (L1 + 2 L2), against the dp4a
      multiply-add rate.
    gemm: 2 M N K G flops of the G plane products, against the measured bf16
      tensor peak (the integer planes are exact bf16 operands); the sustained
      peak where the timed region is seconds long (`sustained`).
    crt (CUDA-core CRT): the 32 x 32 -> 64-bit multiply-adds of
      sum_l v_l M_l, L per output and digit of M_l: M N L ceil(bits(P)/32),
      against the IMAD.WIDE rate.
    crt_sums (tensor-core CRT): the exact bf16 products of the column sums
      Y = V B that are formed, 2 M N (2L) (np - 32 s) flops with np 7-bit
      pieces of P and s groups of 32 not formed (`crt_skip_groups`: below the
      long finish's fast form), against the bf16 tensor peak.
    crt_finish (after the sums): the bytes it moves, the group words formed
      (9 per group of 32 pieces), the 4-byte quotient estimate and the
      output (8 nl + 5 bytes), against HBM.
    scan: the bytes of the two exponent vectors' inputs, against HBM.

    Every stage also carries ``hbm``: its algorithmic bytes (what it must read
    and write once) over its time, against the measured HBM copy rate, whatever
    its own bound: residues read the inputs (8 nl + 5 bytes per entry) and
    write the G planes at `plane_bytes` per entry (2: bf16 planes); the GEMM
    reads both plane stacks and writes the L 16-bit values v_l; the CRT reads
    v_l and writes C (8 nl + 5 bytes per output), the tensor-core sums writing
    the 9-word group sums and the 4-byte estimate in between.
    """
    peaks, src = load_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    L, L1, G, t = info["L"], info["L1"], info["G"], info["t"]
    L2 = L - L1
    md = info["crt_digits"] - 2
    traffic = NCU_TRAFFIC.get(workload, {})
    tkey = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in peaks else "bf16_tflops"
    tpk = float(peaks[tkey])
    tsrc = f"{tkey} ({'sustained, timed region > 1 s' if tkey.endswith('sustained') else 'burst'}), {src}"
    out = {}

    def alu(name, kernel, ops, rate, what):
        ach = ops / (stages[name] / 1e3) / 1e12
        out[name] = {"kernel": kernel, "bound": "alu", "achieved": round(ach, 2),
                     "peak": round(rate / 1e12, 2), "unit": f"T{what}/s", "frac": round(ach * 1e12 / rate, 4),
                     "peak_source": f"{SMS} SMs x {rate / SMS / clk:.0f} {what}/SM/clk x "
                                    f"{clk / 1e6:.0f} MHz (derived)",
                     "traffic": traffic.get(name)}

    res_macs = (M + N) * K * math.ceil((t + 1) / 8) * (L1 + 2 * L2)
    if info.get("res_mode") == 2:
        # the byte products on the tensor cores: 2 flops per byte multiply-add
        ach = 2.0 * res_macs / (stages["residues"] / 1e3) / 1e12
        out["residues"] = {"kernel": "k_residue_mm (integerize + residues as an exact f16 byte GEMM, kind::f16 rate)",
                           "bound": "tensor", "achieved": round(ach, 1), "peak": tpk, "unit": "TFLOP/s",
                           "frac": round(ach / tpk, 4), "peak_source": tsrc, "traffic": traffic.get("residues")}
    else:
        alu("residues", "k_residue (integerize + byte-table residues + plane writes)", res_macs,
            SMS * DP4A_MACS_PER_SM_CLK * clk, "byteMAC")
    if "crt" in stages:
        alu("crt", "k_crt1 / k_crt (direct CRT sum + quotient correction + rounding)", M * N * L * md,
            SMS * IMAD_WIDE_PER_SM_CLK * clk, "imad64")
    if "crt_sums" in stages:
        np_ = info["crt_pieces"] - 32 * info.get("crt_skip_groups", 0)
        fl = 2.0 * M * N * (2 * L) * np_
        ach = fl / (stages["crt_sums"] / 1e3) / 1e12
        out["crt_sums"] = {"kernel": "k_crt_mm (CRT column sums as an exact bf16 GEMM + group carries)",
                           "bound": "tensor", "achieved": round(ach, 1), "peak": tpk, "unit": "TFLOP/s",
                           "frac": round(ach / tpk, 4), "peak_source": tsrc,
                           "traffic": traffic.get("crt_sums")}
        D = info["crt_digits"]
        nl = -(-p // 64)
        ngrp = -(-(info["crt_pieces"] + 5) // 32) - info.get("crt_skip_groups", 0)
        fb = M * N * (4 * 9 * ngrp + 4 + 8 * nl + 5)
        ach = fb / (stages["crt_finish"] / 1e3) / 1e9
        pk = float(peaks["hbm_gbs"])
        out["crt_finish"] = {"kernel": f"{finish_kernel(D)} (CRT finish from the group sums + rounding)",
                             "bound": "hbm", "achieved": round(ach, 1), "peak": pk, "unit": "GB/s",
                             "frac": round(ach / pk, 4), "peak_source": f"hbm_gbs, {src}",
                             "traffic": traffic.get("crt_finish")}
    flops = 2.0 * M * N * K * G
    ach = flops / (stages["gemm"] / 1e3) / 1e12
    out["gemm"] = {"kernel": "k_gemm_tc (plane GEMMs + fused mod-reduce)", "bound": "tensor",
                   "achieved": round(ach, 1), "peak": tpk, "unit": "TFLOP/s", "frac": round(ach / tpk, 4),
                   "peak_source": tsrc, "traffic": traffic.get("gemm")}
    scan_bytes = (M * K + K * N) * (8 + 4)      # top limb + exponent of every entry
    ach = scan_bytes / (stages["scan"] / 1e3) / 1e9
    pk = float(peaks["hbm_gbs"])
    out["scan"] = {"kernel": "k_scan (shared exponents)", "bound": "hbm", "achieved": round(ach, 1),
                   "peak": pk, "unit": "GB/s", "frac": round(ach / pk, 4),
                   "peak_source": f"hbm_gbs, {src}", "traffic": traffic.get("scan")}
    nl = -(-p // 64)
    Kp = -(-K // 8) * 8
    pb = int(info.get("plane_bytes", 2))
    io_in = (M * K + K * N) * (8 * nl + 5)
    c_out = M * N * (8 * nl + 5)
    v_bytes = L * M * N * 2
    nbytes = {"scan": (M * K + K * N) * (8 + 4),
              "residues": io_in + G * (M + N) * Kp * pb,
              "gemm": G * (M + N) * Kp * pb + v_bytes,
              "crt": v_bytes + c_out}
    if "crt_sums" in stages:
        ngrp = -(-(info["crt_pieces"] + 5) // 32) - info.get("crt_skip_groups", 0)
        nbytes["crt_sums"] = v_bytes + M * N * (ngrp * 9 * 4 + 4)
        nbytes["crt_finish"] = M * N * (4 * 9 * ngrp + 4) + c_out
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

class Gpu:
    """Device, launch stream, L2 flush buffer and a CUDA-event timer."""

    def __init__(self, local: int):
        import torch
        self.torch = torch
        torch.cuda.set_device(local)
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.current_stream(self.dev)
        self.flush = torch.empty(512 << 20, dtype=torch.uint8, device=self.dev)

    def timed(self, fn, steps: int, warm: int, each=None):
        """Mean CUDA-event time (ms) of fn over `steps` calls after `warm`
        untimed ones; L2 flushed before every timed call, outside the events."""
        torch = self.torch
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for s_, (a, b) in enumerate(ev):
            self.flush.fill_(s_ & 0xff)
            a.record(self.stream)
            fn()
            b.record(self.stream)
            if each is not None:
                each()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps


def _plan_stages(plan, samples):
    med = {k: statistics.median(s_[k] for s_ in samples) for k in samples[0]}
    info = dict(plan.info)
    if info["crt_mode"] == 2:        # two kernels: the sums on the tensor cores, then the finish
        stages = {k: med[k] for k in ("scan", "residues", "gemm", "crt_sums", "crt_finish")}
        Pm = 1
        for m in plan.moduli():
            Pm *= m
        info["crt_pieces"] = (Pm.bit_length() + 6) // 7 + 1
    else:
        stages = {k: med[k] for k in ("scan", "residues", "gemm", "crt")}
    return stages, info


def measure_single(g: Gpu, ozk, name: str, steps: int, warmup: int, world: int = 1, e2e: bool = True,
                   barrier=None, host=None, **plan_kw):
    """Device-resident (and optionally end-to-end) 2MNK/s of one product
    workload, with the per-stage roofline objects."""
    import synth
    M, N, K, p, (lo, hi), seed = WORKLOADS[name]
    A, B = host if host is not None else synth.workload_single(M, N, K, p, lo, hi, seed)
    dA, dB = ozk.MPMatrix.from_host(A, g.dev), ozk.MPMatrix.from_host(B, g.dev)
    dC = ozk.MPMatrix.empty(M, N, p, g.dev)
    plan = ozk.Plan((M, N, K, p), timing=1, **plan_kw)
    ws = plan.workspace(g.dev)
    samples = []
    barrier = barrier or (lambda: None)
    barrier()
    ms = g.timed(lambda: plan.execute(dA, dB, dC, ws), steps, warmup,
                 each=lambda: samples.append({**plan.timings(), **plan.crt_split()}))
    plan.check()
    barrier()
    ms = max_over_ranks(ms, g.dev)
    work = 2.0 * M * N * K
    res = {"M": M, "N": N, "K": K, "p": p, "ms": ms, "value": replica_value(world, work, ms),
           "plan": plan, "info": dict(plan.info), "samples": samples}
    if e2e:
        res["e2e"] = measure_e2e(g, ozk, plan, A, B, (dA, dB, dC), ws, steps, world, barrier)
    stages, info = _plan_stages(plan, samples)
    sustained = steps * ms / 1e3 > SUSTAINED_AFTER_S
    res["stages"] = stages
    res["kernels"] = stage_rooflines(info, M, N, K, p, stages, name, sustained)
    res["gemm_tflops"] = 2.0 * M * N * K * info["G"] / (stages["gemm"] / 1e3) / 1e12
    res["launches"] = plan.launches()
    del dA, dB, dC, ws
    return res


def host_link_rates(torch, dev, stream, nbytes: int = 1 << 30, reps: int = 3):
    """This box's pinned host <-> device copy rates (GB/s, best of a few
    copies of one buffer each way, CUDA events on the copy stream), reported
    beside the end-to-end figure, which they bound from below."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {}
    for name in ("h2d", "d2h"):
        best = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                if name == "h2d":
                    d.copy_(h, non_blocking=True)
                else:
                    h.copy_(d, non_blocking=True)
                e1.record(stream)
            e1.synchronize()
            best = max(best, nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
        out[name] = round(best, 1)
    out["how"] = "one 1 GiB pinned buffer each way, best of 3 copies"
    del h, d
    return out


def measure_e2e(g: Gpu, ozk, plan, A, B, bufs, ws, steps, world, barrier):
    """End to end through the C ABI: pinned host inputs copied in and the
    result copied out every step, double-buffered on two copy streams so that
    the copies of step s + 1 and s - 1 overlap the product of step s; the timed
    region runs from before the first input copy to after the last output copy."""
    import numpy as np
    torch = g.torch
    dev, stream = g.dev, g.stream
    dA, dB, dC = bufs
    M, N = dC.shape
    p = dC.p

    def pinned(m):
        return {k: torch.from_numpy(np.ascontiguousarray(m[k]).view(np.int64) if k == "limbs" else
                                    np.ascontiguousarray(m[k])).pin_memory() for k in ("limbs", "exp", "sign")}

    hA, hB = pinned(A), pinned(B)
    hC = [{"limbs": torch.empty(dC.limbs.shape, dtype=torch.int64).pin_memory(),
           "exp": torch.empty(dC.exp.shape, dtype=torch.int32).pin_memory(),
           "sign": torch.empty(dC.sign.shape, dtype=torch.int8).pin_memory()} for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in list(hA.values()) + list(hB.values()))
    d2h = sum(v.numel() * v.element_size() for v in hC[0].values())
    bufA = [dA, ozk.MPMatrix.empty(*dA.shape, dA.p, dev)]
    bufB = [dB, ozk.MPMatrix.empty(*dB.shape, dB.p, dev)]
    bufC = [dC, ozk.MPMatrix.empty(M, N, p, dev)]
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
                hC[b][k].copy_(getattr(bufC[b], k), non_blocking=True)
            ev_out[b].record(s_out)

    link = host_link_rates(torch, dev, s_in)
    barrier()
    torch.cuda.synchronize()
    t0.record(s_in)
    copy_in(0)
    for st in range(steps):
        b = st & 1
        if st + 1 < steps:
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
    plan.check()
    e2e_ms = max_over_ranks(t0.elapsed_time(t1) / steps, dev)
    work = 2.0 * M * N * dA.shape[1]
    return {"value": replica_value(world, work, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "copies": "pinned host buffers, every step, double-buffered on two copy streams",
            "host_link_gbs": link}


def measure_batched(g: Gpu, ozk, steps: int = 5, warmup: int = 3, tune: bool = True):
    """64 problems: one CUDA graph of the grouped launches, the grouped
    executes without the graph, and the plain form (one GEMM launch per
    modulus per problem) on the same inputs."""
    import synth
    probs = synth.batched_problems(64, 1002)
    shapes = [(M, N, K, p) for (M, N, K, p, _, _) in probs]
    trip = [(ozk.MPMatrix.from_host(A, g.dev), ozk.MPMatrix.from_host(B, g.dev), ozk.MPMatrix.empty(M, N, p, g.dev))
            for (M, N, K, p, A, B) in probs]
    work = sum(2.0 * M * N * K for (M, N, K, p) in shapes)
    plan_g = ozk.Plan(shapes)
    ws_g = plan_g.workspace(g.dev)
    s = g.torch.cuda.Stream(g.dev)
    with g.torch.cuda.stream(s):
        graph = plan_g.graph(trip, ws_g, s)
    ms_graph = g.timed(lambda: graph.launch(g.stream), steps, warmup)
    ms_grouped = g.timed(lambda: plan_g.execute_batched(trip, ws_g, g.stream), steps, warmup)
    plan_g.check()
    del graph, ws_g
    g.torch.cuda.empty_cache()
    plan_p = ozk.Plan(shapes, schedule=1)
    ws_p = plan_p.workspace(g.dev)
    ms_plain = g.timed(lambda: plan_p.execute_batched(trip, ws_p, g.stream), max(2, steps // 2), warmup)
    plan_p.check()
    del ws_p
    g.torch.cuda.empty_cache()
    out = {"problems": 64, "M_N_K": "log-uniform [128, 2048]", "p": [113, 256, 512],
           "value": work / (ms_graph / 1e3), "unit": UNIT, "graph_ms": ms_graph, "grouped_ms": ms_grouped,
           "plain_ms": ms_plain, "speedup_vs_plain": ms_plain / ms_graph,
           "plain": "one plane-GEMM launch per modulus per problem (other stages grouped)"}
    if tune:
        # autotuned: per-problem K chunk and engines per class, the launch-wide
        # tile measured on the batch; then one CUDA graph of the tuned plan
        import tempfile
        from paper_2609_27831_gb300 import autotune as at
        t0 = time.perf_counter()
        with tempfile.TemporaryDirectory() as td:
            tuned = at.tune_batched(shapes, os.path.join(td, "tune.json"), reps=1)
        tune_s = time.perf_counter() - t0
        plan_t = ozk.Plan(shapes, per_problem=tuned["per_problem"], **tuned["opts"])
        ws_t = plan_t.workspace(g.dev)
        with g.torch.cuda.stream(s):
            graph_t = plan_t.graph(trip, ws_t, s)
        ms_tuned = g.timed(lambda: graph_t.launch(g.stream), steps, warmup)
        plan_t.check()
        del graph_t, ws_t
        g.torch.cuda.empty_cache()
        out.update({"tuned_graph_ms": ms_tuned, "tuned_value": work / (ms_tuned / 1e3),
                    "tuned_speedup_vs_plain": ms_plain / ms_tuned, "tuned_opts": tuned["opts"],
                    "tuned_per_problem_distinct": sorted({json.dumps(d, sort_keys=True)
                                                          for d in tuned["per_problem"]}),
                    "tuning_s": round(tune_s, 1)})
    return out


def measure_complex(g: Gpu, ozk, steps: int = 20, warmup: int = 3, n: int = 1024, p: int = 256):
    """A complex product (Ar + i Ai)(Br + i Bi), 3M form in the residue domain,
    against the four real products of the 4M form on the same parts."""
    import synth
    rng = __import__("numpy").random.Generator(__import__("numpy").random.PCG64(1005))
    parts = [synth.mp_matrix(rng, n, n, p, -32, 32) for _ in range(4)]
    Ar, Ai, Br, Bi = (ozk.MPMatrix.from_host(x, g.dev) for x in parts)
    Cr, Ci = ozk.MPMatrix.empty(n, n, p, g.dev), ozk.MPMatrix.empty(n, n, p, g.dev)
    plan = ozk.ComplexPlan((n, n, n, p))
    ws = plan.workspace(g.dev)
    ms3 = g.timed(lambda: plan.execute_complex(Ar, Ai, Br, Bi, Cr, Ci, ws), steps, warmup)
    plan.check()
    real = ozk.Plan((n, n, n, p))
    wr = real.workspace(g.dev)

    def four():
        for a, b in ((Ar, Br), (Ai, Bi), (Ar, Bi), (Ai, Br)):
            real.execute(a, b, Cr, wr)
    ms4 = g.timed(four, steps, warmup)
    del ws, wr
    g.torch.cuda.empty_cache()
    return {"M": n, "N": n, "K": n, "p": p, "ms_3m": ms3, "ms_four_real_products": ms4,
            "speedup": ms4 / ms3, "value": 4 * 2.0 * n ** 3 / (ms3 / 1e3), "unit": "real 2MNK/s",
            "note": "3M in the residue domain: three plane products per modulus and one CRT per part; "
                    "the comparison runs the four real products (their rounded results do not combine "
                    "exactly)"}


def measure_autograd(g: Gpu, steps: int = 5, warmup: int = 3, n: int = 4096):
    """binary64 forward C = AB and backward dA, dB (three products)."""
    import synth
    from paper_2609_27831_gb300 import autograd as ag
    torch = g.torch
    X, Y, G = synth.fp64_workload(n, 1003)
    xa = torch.tensor(X, device=g.dev, requires_grad=True)
    ya = torch.tensor(Y, device=g.dev, requires_grad=True)
    gt = torch.tensor(G, device=g.dev)

    def step():
        xa.grad = None
        ya.grad = None
        ag.ozaki_matmul(xa, ya).backward(gt)
    ms = g.timed(step, steps, warmup)
    return {"M": n, "N": n, "K": n, "p": 53, "ms_per_step": ms, "value": 3 * 2.0 * n ** 3 / (ms / 1e3),
            "unit": UNIT, "step": "forward C = AB and backward dA, dB (3 products)"}


def measure_int8_peak(g: Gpu, ozk):
    """INT8 tensor-core peak of this GPU: the library's mma.sync s8 probe and
    the library INT8 GEMM behind torch._int_mm (cuBLASLt) at 8192^3."""
    import ctypes as C
    torch = g.torch
    sink = torch.zeros(1, dtype=torch.int32, device=g.dev)
    tops = C.c_double()
    probe = []
    for _ in range(3):
        ozk.check(ozk.lib().ozaki2_probe_mma_s8(SMS * 8, 4096, sink.data_ptr(), C.byref(tops),
                                                g.stream.cuda_stream), "ozaki2_probe_mma_s8")
        probe.append(tops.value)
    out = {"mma_sync_s8_tops": round(max(probe), 1),
           "mma_sync_s8": "m16n8k32 s8 x s8 -> s32, register operands, 8 warps x 8 blocks per SM"}
    try:
        n = 8192
        a = torch.randint(-127, 128, (n, n), dtype=torch.int8, device=g.dev)
        b = torch.randint(-127, 128, (n, n), dtype=torch.int8, device=g.dev)
        ms = g.timed(lambda: torch._int_mm(a, b), 10, 3)
        out["int_mm_tops"] = round(2.0 * n ** 3 / (ms / 1e3) / 1e12, 1)
        out["int_mm"] = "torch._int_mm (cuBLASLt INT8, library) 8192^3"
        del a, b
    except (RuntimeError, AttributeError) as exc:     # not available on this build
        out["int_mm_tops"] = None
        out["int_mm"] = f"unavailable: {str(exc).splitlines()[0][:120]}"
    cands = [v for v in (out["mma_sync_s8_tops"], out["int_mm_tops"]) if v]
    out["int8_peak_tops"] = max(cands)
    # binary64 matrix products (the paper's DGEMM backend runs its moduli on them)
    n = 4096
    x = torch.randn(n, n, dtype=torch.float64, device=g.dev)
    y = torch.randn(n, n, dtype=torch.float64, device=g.dev)
    ms = g.timed(lambda: torch.matmul(x, y), 3, 2)
    out["fp64_matmul_tflops"] = round(2.0 * n ** 3 / (ms / 1e3) / 1e12, 2)
    out["fp64_matmul"] = "torch.matmul float64 (library) 4096^3"
    del x, y
    return out


def _single_summary(r):
    st = r["stages"]
    gk = r["kernels"]["gemm"]
    return {"ms_per_step": r["ms"], "value": r["value"], "unit": UNIT,
            "config": {"M": r["M"], "N": r["N"], "K": r["K"], "p": r["p"], "t": r["info"]["t"],
                       "moduli": r["info"]["L"], "gemms": r["info"]["G"],
                       "plane_groups": r["info"]["plane_groups"], "group_planes": r["info"]["group_planes"],
                       "workspace_gb": round(r["plan"].workspace_bytes / 1e9, 2)},
            "stage_ms": {k: round(v, 4) for k, v in st.items()},
            "plane_gemm_tflops": round(r["gemm_tflops"], 1), "plane_gemm_frac": gk["frac"],
            "plane_gemm_peak": gk["peak_source"]}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import synth
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as ozk

    world, rank, local = dist_info()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    name = args.workload
    M, N, K, p, (lo, hi), seed = WORKLOADS[name]
    A, B = synth.workload_single(M, N, K, p, lo, hi, seed)
    # the CPU baseline's spawn pool: the oracle on sampled entries of the same workload
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ot = OracleTimer(A, B, K)
        rate, n_ent, wall = ot.rate()
        ot.close()
        cpu = {"value": rate, "unit": UNIT, "cores": ot.cores, "kind": "oracle",
               "sample": f"oracle ozaki2_entries (stage-by-stage method, exact integers) on {n_ent} sampled "
                         f"output entries of the {M}x{N}x{K} p={p} workload, each a full K={K} inner product; "
                         f"spawn pool of {ot.cores} processes; wall {wall:.1f} s; rate = 2K per entry / wall"}
    g = Gpu(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=g.dev)

    def barrier():
        if world > 1:
            dist.barrier()

    props = torch.cuda.get_device_properties(g.dev)
    uuid = getattr(props, "uuid", None)
    clk = ClockSampler(f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-")
                       else (str(uuid) if uuid is not None else local))
    clk.start()
    r = measure_single(g, ozk, name, args.steps, args.warmup, world, e2e=not args.no_e2e, barrier=barrier,
                       host=(A, B))
    clocks = clk.stop()
    stages, kernels = r["stages"], r["kernels"]
    dom = max(stages, key=stages.get)
    roof = dict(kernels[dom])
    roof["stage_ms"] = {k: round(v, 4) for k, v in stages.items()}
    info = r["info"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16-int (exact integer planes on tcgen05 kind::f16)",
        "data": "synthetic", "impl": "ours",
        "config": {"workload": name, "M": M, "N": N, "K": K, "p": p, "exp_range": [lo, hi], "seed": seed,
                   "t": info["t"], "moduli": info["L"], "gemms": info["G"],
                   "plane_groups": info["plane_groups"], "group_planes": info["group_planes"],
                   "workspace_gb": round(r["plan"].workspace_bytes / 1e9, 2),
                   "parallelism": f"replicas{world}",
                   "l2": "flushed (512 MiB write between steps); inputs larger than L2"},
        "roofline": roof,
        "kernels": {k: v for k, v in kernels.items() if k != dom},
        "plane_gemm_tflops": round(r["gemm_tflops"], 1),
        "gpu_launches": r["launches"] * args.steps,
        "clocks": clocks,
    }
    if "e2e" in r:
        line["e2e"] = r["e2e"]
    if cpu is not None:
        line["cpu_baseline"] = cpu
    del r
    torch.cuda.empty_cache()
    if not args.no_sweep and world == 1:
        sweep = {}
        for wl in ("gemm_1024_p256", "gemm_8192_p53", "gemm_256_p53"):
            if wl == name:
                continue
            st_ = {"gemm_1024_p256": 200, "gemm_8192_p53": 5, "gemm_256_p53": 200}[wl]
            rr = measure_single(g, ozk, wl, st_, 5, e2e=False)
            sweep[wl] = _single_summary(rr)
            line["gpu_launches_sweep"] = line.get("gpu_launches_sweep", 0) + rr["launches"] * (st_ + 5)
            del rr
            torch.cuda.empty_cache()
        if info["plane_groups"] > 1:
            # the same product with every plane resident at once (one group)
            rr = measure_single(g, ozk, name, 3, 3, e2e=False, host=(A, B), plane_group=-1)
            sweep[name + "_one_group"] = _single_summary(rr)
            del rr
            torch.cuda.empty_cache()
        sweep["batched64"] = measure_batched(g, ozk)
        sweep["dgemm4096_autograd"] = measure_autograd(g)
        sweep["complex_1024_p256"] = measure_complex(g, ozk)
        i8 = measure_int8_peak(g, ozk)
        G_ = info["G"]
        plane_int = 2.0 * M * N * K * G_ / (stages["gemm"] / 1e3) / 1e12
        i8["plane_gemm_int_tops"] = round(plane_int, 1)
        i8["plane_gemm_frac_of_int8_peak"] = round(plane_int / i8["int8_peak_tops"], 3)
        i8["note"] = ("the plane GEMMs run exact integer products on tcgen05 kind::f16 (bf16 operands, "
                      "fp32 accumulation kept exact by K chunks); their integer-operation rate is stated "
                      "against this GPU's INT8 tensor peak, which is below the bf16 rate")
        # the second plane GEMM engine (INT8 x INT8 -> INT32 on mma.sync) against the default,
        # same product, same bits
        ab = {}
        for eng, label in ((0, "tcgen05_bf16"), (2, "mma_sync_s8")):
            rr = measure_single(g, ozk, "gemm_1024_p256", 20 if eng == 0 else 5, 3, e2e=False, engine=eng)
            gm = rr["stages"]["gemm"]
            ops = 2.0 * 1024 ** 3 * rr["info"]["G"]
            ab[label] = {"gemm_ms": round(gm, 4), "int_tops": round(ops / (gm / 1e3) / 1e12, 1),
                         "frac_of_int8_peak": round(ops / (gm / 1e3) / 1e12 / i8["int8_peak_tops"], 3),
                         "ms_per_step": round(rr["ms"], 4)}
            del rr
            torch.cuda.empty_cache()
        ab["workload"] = "gemm_1024_p256"
        i8["engines"] = ab
        sweep["int8"] = i8
        line["sweep"] = sweep
        line["clocks_sweep_excluded"] = "clocks are sampled over the main workload's timed region"
    del A, B
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    import synth
    name = args.workload
    M, N, K, p, (lo, hi), seed = WORKLOADS[name]
    A, B = synth.workload_single(M, N, K, p, lo, hi, seed)
    ot = OracleTimer(A, B, K)
    del A, B
    for _ in range(args.warmup):
        ot.batch(1)
    rates = []
    n_tot, wall_tot = 0, 0.0
    for _ in range(args.steps):
        n, w = ot.batch(ot.cores)
        rates.append(n * 2.0 * K / w)
        n_tot += n
        wall_tot += w
    ot.close()
    value = statistics.median(rates)
    ms = 2.0 * M * N * K / value * 1e3
    sample = (f"oracle ozaki2_entries on {ot.cores} sampled output entries per step (one per host core, "
              f"full K={K}) of the {M}x{N}x{K} p={p} workload; {n_tot} entries in {wall_tot:.1f} s")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms,
        "ms_per_step_kind": "extrapolated: the whole product's 2MNK at the sampled entries' rate",
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "exact integers (Python)", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": name, "M": M, "N": N, "K": K, "p": p, "exp_range": [lo, hi], "seed": seed,
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ot.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_workload_only(args):
    """One workload's device-resident timing only (for profilers and quick
    checks): no end-to-end leg, no sweep, no CPU baseline."""
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as ozk
    g = Gpu(0)
    if args.workload == "batched64":
        out = measure_batched(g, ozk, args.steps, args.warmup)
    elif args.workload == "dgemm4096_autograd":
        out = measure_autograd(g, args.steps, args.warmup)
    else:
        kw = {"gemm_tile": args.gemm_tile} if args.gemm_tile else {}
        if args.engine:
            kw["engine"] = args.engine
        out = _single_summary(measure_single(g, ozk, args.workload, args.steps, args.warmup, e2e=False, **kw))
    out.update({"metric": METRIC, "workload": args.workload, "steps": args.steps, "warmup": args.warmup,
                "impl": "ours", "only": True})
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + ["batched64", "dgemm4096_autograd"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only", action="store_true",
                    help="time the workload alone (device-resident), e.g. under a profiler")
    ap.add_argument("--gemm-tile", type=int, default=0, choices=[0, 1, 2],
                    help="with --only: plane GEMM tile (0 automatic, 1 one SM, 2 CTA pairs)")
    ap.add_argument("--engine", type=int, default=0, choices=[0, 1, 2],
                    help="with --only: plane GEMM engine (0 tcgen05 bf16, 1 CUDA cores, 2 INT8 mma.sync)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        if args.workload not in WORKLOADS:
            raise SystemExit("the reference arm times single-product workloads")
        run_reference(args)
    elif args.only or args.workload not in WORKLOADS:
        run_workload_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
