"""Throughput of the batched form: the seeded set of 48 uneven replicas
(bcc 3^3..6^3 cells, 0-5 % vacancies, 52 to 432 atoms, mixed fp16, Krylov
rank 6), all stepped together by sxl_batch_step, against the same replicas
stepped one after another (one host thread).  Every replica starts from the
neutral non-magnetic n = 0 history.

    python -m paper_2303_03529_gb300.batch_bench [--steps K] [--warmup W] [--threads T] [--autotune]

Prints one JSON line: replica MD steps/s and atom-steps/s of the batch, the
sequential value, and the tensor-core throughput summed over the replicas.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import sxl, workload


def run(batch, steps, threads):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(steps, nthreads=threads)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--threads", type=int, default=48)
    ap.add_argument("--count", type=int, default=48)
    ap.add_argument("--autotune", action="store_true",
                    help="tile autotuning of every replica before the run")
    ap.add_argument("--recycle", action="store_true",
                    help="the recycled-subspace kernel with fused responses (a variant, "
                         "not the paper's Krylov construction)")
    args = ap.parse_args()
    reps = workload.replica_set(args.count)
    b = sxl.Batch(reps, "fp16", krylov_recycle=1 if args.recycle else 0)
    tuned = b.autotune() if args.autotune else None
    for ctx, w in zip(b.contexts, reps):
        nat = w.R.shape[0]
        ctx.set_state(w.R, w.V, np.zeros((w.params.kmax + 1, 2 * nat)), float("nan"))
    run(b, args.warmup, args.threads)
    for ctx in b.contexts:
        ctx.enable_gemm_timing(True)
        ctx.timers(reset=True)
    t_batch = run(b, args.steps, args.threads)
    tm = [ctx.timers(reset=True) for ctx in b.contexts]
    for ctx in b.contexts:
        ctx.enable_gemm_timing(False)
    t_seq = run(b, args.steps, 1)
    atoms = sum(w.R.shape[0] for w in reps)
    alg = sum(t["tc_alg_flops"] for t in tm)
    out = {
        "metric": f"replica MD steps/s ({len(reps)} replicas, "
                  f"{min(w.R.shape[0] for w in reps)}-{max(w.R.shape[0] for w in reps)} atoms)",
        "value": round(len(reps) * args.steps / t_batch, 3),
        "unit": "replica-steps/s",
        "atom_steps_per_s": round(atoms * args.steps / t_batch, 1),
        "sequential_value": round(len(reps) * args.steps / t_seq, 3),
        "speedup_vs_sequential": round(t_seq / t_batch, 3),
        "host_threads": args.threads,
        "steps": args.steps, "warmup": args.warmup,
        "tensor_tflops_aggregate": round(alg / t_batch / 1e12, 1),
        "gemm_launches": int(sum(t["tc_launches"] for t in tm)),
        "precision": "fp16", "data": "synthetic (workload.replica_set, seeded)",
        "tiles": "autotuned per chain dimension" if tuned else "library defaults",
        "krylov": "recycled subspace, fused responses" if args.recycle else "Krylov construction",
        "tuned": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in t.items()}
                  for t in tuned] if tuned else None,
    }
    print(json.dumps(out), flush=True)
    b.close()


if __name__ == "__main__":
    main()
