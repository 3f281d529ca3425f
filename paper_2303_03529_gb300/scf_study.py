"""SCF-acceleration study of Sec. IV (Fig. SCF) on the GPU.

1. Iterations and wall time to RMS(q - n) < tol for the kernel quasi-Newton
   mixer (Eq. QN), Pulay DIIS and linear mixing (0.06), from the same start:
   the 16-atom cell of the paper's SCF figure in the FP64 form
   (ferromagnetic start, tol 1e-8) and the 1024-atom cell in the mixed fp16
   form (from n = 0, tol 1e-5; the kernel mixer keeps K0 = -I there, since
   the exact K0 would take 2048 responses).
2. Regular BOMD with DIIS-converged forces against sXL-BOMD: wall time per
   MD step at 1024 atoms (fp16), BOMD converging each step to 1e-5.

Prints one JSON line per measurement.

    python -m paper_2303_03529_gb300.scf_study [--quick]
"""
import argparse
import json
import time

import numpy as np
import torch

from . import sxl, workload


def _scf(w, precision, n0, tol, mixer, max_iter, keep_k0):
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, precision, scf_keep_k0=keep_k0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        n, its, rms, hist = ctx.scf_ex(w.R, n0, tol=tol, max_iter=max_iter, mixer=mixer)
        ok = True
    except sxl.SxlError:
        its, rms, hist, ok, n = max_iter, float("nan"), np.array([]), False, None
    dt = time.perf_counter() - t0
    ctx.close()
    return dict(study="scf", workload=w.name, precision=precision, mixer=mixer, tol=tol,
                converged=ok, iterations=int(its), seconds=round(dt, 3),
                rms_history=[float(x) for x in hist[:: max(1, len(hist) // 40)]]), n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="skip the 1024-atom parts")
    ap.add_argument("--md-steps", type=int, default=3)
    args = ap.parse_args()

    w16 = workload.fe16()
    for mixer, cap in (("kernel", 400), ("diis", 400), ("linear", 1500)):
        rec, _ = _scf(w16, "fp64", w16.n0, 1e-8, mixer, cap, 0)
        print(json.dumps(rec), flush=True)
    if args.quick:
        return

    w = workload.fe1024()
    zero = np.zeros(2 * w.n_atoms)
    n_star = None
    for mixer, cap in (("kernel", 100), ("diis", 100), ("linear", 200)):
        rec, n = _scf(w, "fp16", zero, 1e-5, mixer, cap, 1)
        print(json.dumps(rec), flush=True)
        if mixer == "kernel":
            n_star = n

    # BOMD (DIIS, 1e-5 per step) against sXL-BOMD, from the same SCF state
    p = w.params
    nh = torch.stack([n_star] * (p.kmax + 1)).contiguous()
    out = {}
    for kind in ("sxl", "bomd"):
        ctx = sxl.Context(p, w.n_atoms, w.cell, "fp16", scf_keep_k0=1)
        _, mu = ctx.density(w.R, n_star)
        ctx.set_state(w.R, w.V, nh, mu)
        if kind == "sxl":
            ctx.step(1, stats=False)                       # evaluates the state, one warm-up step
        else:
            ctx.bomd(1, tol=1e-5, max_iter=100, mixer="diis", stats=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if kind == "sxl":
            ctx.step(args.md_steps, stats=False)
            its = None
        else:
            _, its = ctx.bomd(args.md_steps, tol=1e-5, max_iter=100, mixer="diis", stats=False)
        torch.cuda.synchronize()
        out[kind] = (time.perf_counter() - t0) / args.md_steps
        print(json.dumps(dict(study="md_step_time", workload=w.name, precision="fp16", kind=kind,
                              steps=args.md_steps, seconds_per_step=round(out[kind], 4),
                              scf_iterations=None if its is None else [int(x) for x in its])),
              flush=True)
        ctx.close()
    print(json.dumps(dict(study="md_step_time_ratio", bomd_over_sxl=round(out["bomd"] / out["sxl"], 3))))


if __name__ == "__main__":
    main()
