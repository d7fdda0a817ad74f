"""Run one named workload a few times (for profilers such as ncu).

    python -m paper_2609_27831_gb300.profile_run --workload gemm_1024_p256 --reps 2
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "gemm_256_p53": (256, 256, 256, 53, -8, 8, 1000),
    "gemm_1024_p256": (1024, 1024, 1024, 256, -32, 32, 1001),
    "gemm_1024_p53": (1024, 1024, 1024, 53, -8, 8, 1001),
    "gemm_2048_p256": (2048, 2048, 2048, 256, -32, 32, 1001),
    "gemm_2048_p512": (2048, 2048, 2048, 512, -8, 8, 1001),
    "gemm_4096_p53": (4096, 4096, 4096, 53, -8, 8, 1001),
    "gemm_1024_p1024": (1024, 1024, 1024, 1024, -64, 64, 1001),
    "gemm_1024_p2048": (1024, 1024, 1024, 2048, -64, 64, 1001),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gemm_1024_p256", choices=sorted(WORKLOADS))
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--schedule", type=int, default=0)
    ap.add_argument("--res-engine", type=int, default=0)
    ap.add_argument("--crt-engine", type=int, default=0)
    ap.add_argument("--time", action="store_true",
                    help="also print the median per-stage milliseconds over --reps timed products")
    args = ap.parse_args()
    import torch

    import synth
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as ozk
    M, N, K, p, lo, hi, seed = WORKLOADS[args.workload]
    A, B = synth.workload_single(M, N, K, p, lo, hi, seed)
    dA, dB = ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B)
    C = ozk.MPMatrix.empty(M, N, p)
    plan = ozk.Plan((M, N, K, p), schedule=args.schedule, res_engine=args.res_engine,
                    crt_engine=args.crt_engine, timing=1 if args.time else 0)
    ws = plan.workspace()
    for _ in range(args.reps):
        plan.execute(dA, dB, C, ws)
    plan.check()
    torch.cuda.synchronize()
    print("ok", args.workload, plan.info)
    if args.time:
        import statistics
        stages = []
        for _ in range(args.reps):
            plan.execute(dA, dB, C, ws)
            stages.append(plan.timings())
        plan.check()
        med = {k: round(statistics.median(t[k] for t in stages), 4) for k in stages[0]}
        print("stage_ms", args.workload, med,
              "rate_2MNK_per_s %.4g" % (2.0 * M * N * K / (med["total"] / 1e3)))


if __name__ == "__main__":
    main()
