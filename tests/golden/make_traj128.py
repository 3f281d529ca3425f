"""Writes tests/golden/fe128_traj_fp64.json: 200 sXL-BOMD steps (Eq.
Integration, dt 0.5 fs, Krylov rank 6) of the seeded 128-atom cell
(workload.fe128) computed by the FP64 oracle alone.

The trajectory starts at the SCF fixed point n* (Eq. QN, converged to
RMS(q - n) < 1e-10 from the ferromagnetic start) with every history slot
n(t0 - k dt) = n* (Sec. II.E) and the preconditioner K0 = J^{-1} evaluated
exactly at n*, the density of the initial time step.  Stored: n*, mu*, the
per-step total energy, temperature, RMS(q - n) and mu, and the full state
(R, V, n) at steps 50, 100 and 200.  The GPU test replays the run from the
same start (tests/test_gpu_traj128.py).

    python tests/golden/make_traj128.py          (about 30 min on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dynamics, electronic, kernel  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402

STEPS = 200
CHECKPOINTS = (50, 100, 200)


def main():
    t0 = time.time()
    w = wl.fe128()
    p = w.params
    scf = dynamics.scf(w.R, w.cell, w.n0, p, tol=1e-10, max_iter=400)
    n_star, mu_star = scf["n"], scf["mu"]
    K0 = kernel.exact_kernel(electronic.density(w.R, w.cell, n_star, p, mu_guess=mu_star))
    md = dynamics.XLBOMD(w.R, w.V, w.cell, n_star, p, K0, mu=mu_star)
    start = md.stats()
    out = {"workload": w.name, "source": "oracle (tests/golden/make_traj128.py)",
           "dt_fs": p.dt_fs, "krylov_rank": p.krylov_rank, "steps": STEPS,
           "scf_iters": scf["iters"], "n_star": n_star.tolist(), "mu_star": mu_star,
           "start": {k: float(v) for k, v in start.items()},
           "stats": {"Etot": [], "T": [], "rms": [], "mu": []}, "checkpoints": {}}
    for s in range(1, STEPS + 1):
        st = md.step()
        for k in out["stats"]:
            out["stats"][k].append(float(st[k]))
        if s in CHECKPOINTS:
            out["checkpoints"][str(s)] = {"R": md.R.tolist(), "V": md.V.tolist(),
                                          "n": md.nhist[0].tolist()}
        if s % 10 == 0:
            print(f"step {s} Etot {st['Etot']:.10f} rms {st['rms']:.2e} "
                  f"({time.time() - t0:.0f} s)", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fe128_traj_fp64.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


if __name__ == "__main__":
    main()
