"""Energy drift of sXL-BOMD at 2000 atoms (bcc 10x10x10, 18000 orbitals x 2
spins, padded to 18048 in the mixed forms): SCF to 1e-5 from n = 0 (kernel
mixer, K0 = -I), then `--steps` MD steps of 0.5 fs with the total energy
taken every `--every` steps; prints the drift (least-squares slope) in
eV/atom/ps and the spread of the energy as one JSON line.

    python -m paper_2303_03529_gb300.drift_run [--steps 100] [--every 10] [--precision fp16]
"""
import argparse
import json
import time

import numpy as np
import torch

from . import sxl, workload


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--precision", default="fp16")
    ap.add_argument("--workload", default="fe2000")
    args = ap.parse_args()
    w = workload.WORKLOADS[args.workload]()
    p = w.params
    ctx = sxl.Context(p, w.n_atoms, w.cell, args.precision, scf_keep_k0=1)
    t0 = time.perf_counter()
    n_star, its, rms = ctx.scf(w.R, np.zeros(2 * w.n_atoms), tol=1e-5, max_iter=60)
    t_scf = time.perf_counter() - t0
    _, mu = ctx.density(w.R, n_star)
    ctx.set_state(w.R, w.V, torch.stack([n_star] * (p.kmax + 1)).contiguous(), mu)
    times, E, T, res = [], [], [], []
    t_md = 0.0
    st = ctx.step(1, stats=True)            # energy at the first step
    done = 1
    times.append(done * p.dt_fs); E.append(st[0, 0]); T.append(st[0, 1]); res.append(st[0, 2])
    while done < args.steps:
        k = min(args.every - 1, args.steps - done - 1)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if k > 0:
            ctx.step(k, stats=False)
        st = ctx.step(1, stats=True)
        torch.cuda.synchronize()
        t_md += time.perf_counter() - t1
        done += k + 1
        times.append(done * p.dt_fs); E.append(st[0, 0]); T.append(st[0, 1]); res.append(st[0, 2])
    tps = np.array(times) / 1000.0
    e_atom = np.array(E) / w.n_atoms
    slope = float(np.polyfit(tps, e_atom, 1)[0]) if len(tps) > 1 else float("nan")
    out = dict(study="drift", workload=w.name, n_atoms=w.n_atoms, precision=args.precision,
               orbitals=9 * w.n_atoms, dt_fs=p.dt_fs, steps=done, scf_iterations=its,
               scf_rms=rms, scf_seconds=round(t_scf, 2),
               seconds_per_step=round(t_md / max(done - 1, 1), 3),
               drift_eV_per_atom_per_ps=slope,
               energy_spread_eV_per_atom=float(e_atom.max() - e_atom.min()),
               T_K_last=float(T[-1]), max_rms_residual=float(max(res)),
               energy_eV_per_atom=[float(x) for x in e_atom])
    print(json.dumps(out), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
