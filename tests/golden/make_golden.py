"""Writes tests/golden/fe16_fp64.json: the oracle's density, response,
shadow energy and forces for the seeded 16-atom cell (workload.fe16, the size
of the paper's Fe supercell, Sec. III.B) at its ferromagnetic start n0, and the
converged SCF fixed point (Eq. QN).  The paper prints no worked numeric
example, so these values come from the oracle alone; they pin the oracle
against accidental change (tests/test_golden.py), not against the paper.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dynamics, electronic, energy, model  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


def main():
    w = wl.fe16()
    d = electronic.density(w.R, w.cell, w.n0, w.params)
    qv, dmu = d.response(wl.random_direction(w.n_atoms, 11))
    H0 = model.build_h0(w.R, w.cell, w.params)
    e = energy.shadow_energy(d, H0, model.repulsive_energy(w.R, w.cell, w.params))
    F = energy.forces(d, w.R, w.cell)
    scf = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-10)
    out = {
        "workload": w.name, "source": "oracle (tests/golden/make_golden.py)",
        "mu": d.mu, "q": d.q.tolist(), "spin": d.spin.tolist(),
        "response_direction_seed": 11, "qv": qv.tolist(), "dmu": dmu,
        "energies": {k: float(v) for k, v in e.items()},
        "forces": F.tolist(),
        "scf_n": scf["n"].tolist(), "scf_mu": scf["mu"], "scf_iters": scf["iters"],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fe16_fp64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
