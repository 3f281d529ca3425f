"""The plain FP64 form at the benchmark's size (1024 atoms, 9216 orbitals x 2
spins): one density (Fermi-operator expansion with the common-mu Newton
search to |N - N_e| < 1e-10), one Krylov response direction and the forces,
each timed on the device (CUDA events on the context stream), with the fp64
GEMM launches and their rate from the library's per-form counters.

A full FP64 MD step is one such density, `krylov_rank` responses and the
forces; the step time printed is that sum.  The density starts from the
chemical potential the fp16 form finds for the same state (one pass
suffices for it), so the count of FP64 passes is what an MD step with a
good extrapolated start needs.

With --oracle the FP64 result is also compared with the oracle (dense
eigendecomposition on the host cores): charges, mu, the response and the
forces.

    python -m paper_2303_03529_gb300.fp64_study [--oracle]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import build, sxl, workload


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="fe1024")
    ap.add_argument("--oracle", action="store_true")
    args = ap.parse_args()
    build.build()
    torch.cuda.set_device(0)
    w = workload.WORKLOADS[args.workload]()
    p, nat = w.params, w.n_atoms
    n0 = np.zeros(2 * nat)
    v = workload.random_direction(nat, 21)
    # starting mu from the fp16 form (seconds)
    c16 = sxl.Context(p, nat, w.cell, "fp16", scf_keep_k0=1)
    _, mu16 = c16.density(w.R, n0)
    c16.close()
    ctx = sxl.Context(p, nat, w.cell, "fp64", scf_keep_k0=1)
    ctx.enable_gemm_timing(True)
    st = torch.cuda.current_stream()
    out = {"workload": w.name, "n_atoms": nat, "orbitals": w.n_orb, "mu_start_fp16": mu16}

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    g0 = ctx.info()["gemms"]
    (q, mu), t_d = timed(lambda: ctx.density(w.R, n0, mu16))
    info = ctx.info()
    out["density"] = {"s": round(t_d, 2), "mu": mu, "foe_steps": int(info["foe_steps"]),
                      "gemm_launches": int(info["gemms"] - g0)}
    g0 = info["gemms"]
    (qv, dmu), t_r = timed(lambda: ctx.response(v))
    out["response"] = {"s": round(t_r, 2), "gemm_launches": int(ctx.info()["gemms"] - g0)}
    # forces at the same state (the call repeats the density: its own time
    # minus the density's is the force kernel's)
    (F, _), t_f = timed(lambda: ctx.forces(w.R, n0, energies=False))
    out["forces_incl_density_s"] = round(t_f, 2)
    gt = ctx.gemm_timers(reset=True)["fp64"]
    out["fp64_gemm"] = {"launches": int(gt["launches"]), "ms": round(gt["ms"], 1),
                        "tflops": round(gt["product_flops"] / (gt["ms"] / 1e3) / 1e12, 3)}
    m = p.krylov_rank
    step = t_d + m * t_r + max(t_f - t_d, 0.0)
    out["md_step_estimate_s"] = round(step, 1)
    out["md_steps_per_s"] = round(1.0 / step, 6)
    if args.oracle:
        from oracle import electronic, energy
        t0 = time.perf_counter()
        d = electronic.density(w.R, w.cell, n0, p)
        qv_o, _ = d.response(v)
        F_o = energy.forces(d, w.R, w.cell)
        out["oracle"] = {"s": round(time.perf_counter() - t0, 1),
                         "max_dq": float(np.abs(q.cpu().numpy() - d.q).max()),
                         "dmu": float(abs(mu - d.mu)),
                         "max_dqv": float(np.abs(qv.cpu().numpy() - qv_o).max()),
                         "max_dF": float(np.abs(F.cpu().numpy() - F_o).max())}
    ctx.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
