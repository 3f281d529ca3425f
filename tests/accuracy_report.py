"""Accuracy of the mixed-precision forms against the FP64 form and the oracle.

    python tests/accuracy_report.py [--steps 200] [--skip-1024]

1. 128-atom cell: one SCF point (FP64, exact K0), then the same sXL-BOMD
   trajectory (K0 = -I, rank 6, dt 0.5 fs) in the FP64, fp16 and bf16 forms.
   Trajectories of different precision drift apart, so q, m, F and U are
   compared at equal states: every 10 steps each form evaluates the FP64
   trajectory's (R, n).  Also the total-energy drift of each form's own
   trajectory (linear fit, eV/atom/ps) and its RMS fluctuation.
2. 1024-atom cell (the benchmark workload): one evaluation at (R, n = 0) in
   fp16 and bf16 against the FP64 oracle (dense eigendecomposition): mu, q,
   m, the energy terms and the forces.
Prints one JSON document.  It uses the oracle as the reference, so it lives
with the tests; it is a measurement script, not part of the library.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def drift_per_atom_ps(E, dt_fs, nat):
    import numpy as np
    t = np.arange(len(E)) * dt_fs * 1e-3  # ps
    slope = np.polyfit(t, E, 1)[0]
    return float(slope / nat), float(np.std(E - np.polyval(np.polyfit(t, E, 1), t)) / nat)


def part128(steps):
    import numpy as np
    from paper_2303_03529_gb300 import sxl, workload
    w = workload.fe128()
    p = w.params
    h = w.n_atoms
    ref = sxl.Context(p, w.n_atoms, w.cell, "fp64")
    n_star, iters, rms = ref.scf(w.R, w.n0, tol=1e-9, max_iter=300)
    _, mu0 = ref.density(w.R, n_star)
    nh = np.tile(n_star.cpu().numpy(), (p.kmax + 1, 1))
    out = {"scf": {"iters": iters, "rms": rms}, "steps": steps, "dt_fs": p.dt_fs}
    trajs = {k: sxl.Context(p, w.n_atoms, w.cell, k) for k in ("fp64", "fp16", "bf16")}
    for c in trajs.values():
        c.set_state(w.R, w.V, nh, mu0)
    # separate contexts evaluate every form at the FP64 trajectory's states
    probe = {k: sxl.Context(p, w.n_atoms, w.cell, k) for k in ("fp64", "fp16", "bf16")}
    stats = {k: [] for k in trajs}
    errs = {"fp16": [], "bf16": []}
    wall = {k: 0.0 for k in trajs}
    for s0 in range(0, steps, 10):
        R, V, nhist, mu = trajs["fp64"].get_state()
        n = nhist[0].contiguous()
        F64, e64 = probe["fp64"].forces(R, n)
        q64, _ = probe["fp64"].density(R, n)
        for k in errs:
            F, e = probe[k].forces(R, n)
            q, _ = probe[k].density(R, n)
            qq, qq64 = q.cpu().numpy(), q64.cpu().numpy()
            errs[k].append({"dq": float(np.abs(qq - qq64).max()),
                            "dm": float(np.abs((qq[:h] - qq[h:]) - (qq64[:h] - qq64[h:])).max()),
                            "dF": (F - F64).abs().max().item(),
                            "dU_per_atom": abs(e["U"] - e64["U"]) / h,
                            "dEband_per_atom": abs(e["band"] - e64["band"]) / h})
        for k, c in trajs.items():
            t0 = time.time()
            stats[k].append(c.step(min(10, steps - s0)))
            wall[k] += time.time() - t0
    for k in trajs:
        st = np.concatenate(stats[k])
        d, fl = drift_per_atom_ps(st[:, 0], p.dt_fs, h)
        out[k] = {"drift_eV_per_atom_ps": d, "fluct_eV_per_atom": fl,
                  "T_end_K": float(st[-1, 1]), "rms_residual_max": float(st[:, 2].max()),
                  "wall_s": round(wall[k], 1)}
    for k, v in errs.items():
        out[k]["vs_fp64_at_fp64_states_max"] = {f: max(x[f] for x in v) for f in v[0]}
    return out


def part1024():
    import numpy as np
    from oracle import electronic, energy, model
    from paper_2303_03529_gb300 import sxl, workload
    w = workload.fe1024()
    p = w.params
    n = np.zeros(2 * w.n_atoms)
    t0 = time.time()
    d = electronic.density(w.R, w.cell, n, p)
    H0 = model.build_h0(w.R, w.cell, p)
    e_o = energy.shadow_energy(d, H0, model.repulsive_energy(w.R, w.cell, p))
    F_o = energy.forces(d, w.R, w.cell)
    t_oracle = time.time() - t0
    out = {"oracle_s": round(t_oracle, 1)}
    for prec in ("fp16", "bf16"):
        ctx = sxl.Context(p, w.n_atoms, w.cell, prec)
        q, mu = ctx.density(w.R, n)
        F, e = ctx.forces(w.R, n)
        q = q.cpu().numpy()
        h = w.n_atoms
        out[prec] = {
            "dmu_eV": abs(mu - d.mu),
            "dq": float(np.abs(q - d.q).max()),
            "dm": float(np.abs((q[:h] - q[h:]) - d.spin).max()),
            "dF_eV_per_A": float(np.abs(F.cpu().numpy() - F_o).max()),
            "dU_per_atom": abs(e["U"] - e_o["U"]) / h,
            "dEband_per_atom": abs(e["band"] - e_o["band"]) / h,
            "dEentropy_per_atom": abs(e["entropy"] - e_o["entropy"]) / h,
            "foe_steps": ctx.info()["foe_steps"]}
        ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--skip-1024", action="store_true")
    args = ap.parse_args()
    from paper_2303_03529_gb300 import build
    build.build()
    rep = {"fe128": part128(args.steps)}
    if not args.skip_1024:
        rep["fe1024"] = part1024()
    print(json.dumps(rep, indent=1))


if __name__ == "__main__":
    main()
