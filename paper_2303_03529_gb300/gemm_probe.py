"""Times the tensor-core GEMM of the mixed-precision chains in isolation.

    python -m paper_2303_03529_gb300.gemm_probe --n 4608 --reps 5 [--bf16] [--plain] [--sym]

n must be 9 N_at with N_at a multiple of 64 (n = 576, 1152, ..., 9216).  The
product C = A B^T of two random (2 x n x n) operands runs through the
library's sxl_mixed_gemm; the kernel's own device time comes from the
library's CUDA-event counters (sxl_timers), so the fp64 -> (hi, lo)
conversions around it are not counted.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4608)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--bf16", action="store_true")
    ap.add_argument("--plain", action="store_true")
    ap.add_argument("--sym", action="store_true")
    args = ap.parse_args()
    import torch
    from . import build, sxl, workload

    build.build()
    n = args.n
    assert n % 576 == 0, "n must be 9 N_at with N_at a multiple of 64"
    ctx = sxl.Context(workload.ModelParams(), n // 9, [60.0, 60.0, 60.0],
                      "bf16" if args.bf16 else "fp16")
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(2, n, n, generator=g, device="cuda", dtype=torch.float64) / n ** 0.5
    B = A if args.sym else torch.randn(2, n, n, generator=g, device="cuda",
                                       dtype=torch.float64) / n ** 0.5
    ctx.mixed_gemm(A, B, sym=args.sym, split=not args.plain)  # warm-up
    ctx.enable_gemm_timing(True)
    ctx.timers(reset=True)
    for _ in range(args.reps):
        ctx.mixed_gemm(A, B, sym=args.sym, split=not args.plain)
    t = ctx.timers(reset=True)
    ms = t["tc_ms"] / t["tc_launches"]
    print(json.dumps({
        "n": n, "split": not args.plain, "sym": args.sym, "bf16": args.bf16,
        "launches": int(t["tc_launches"]), "ms_per_launch": round(ms, 4),
        "tensor_tflops": round(t["tc_alg_flops"] / t["tc_launches"] / ms / 1e9, 1),
        "mma_issued_tflops": round(t["tc_mma_flops"] / t["tc_launches"] / ms / 1e9, 1),
        "fp32_equiv_tflops": round(t["tc_fp32_flops"] / t["tc_launches"] / ms / 1e9, 1)}))
    ctx.close()


if __name__ == "__main__":
    main()
