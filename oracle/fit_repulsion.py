"""Fit of the pair-repulsion prefactor A of the synthetic model.

Test infrastructure only (see oracle/__init__.py).  Run as
``python -m oracle.fit_repulsion``; it prints the value stored as
ModelParams.rep_A in paper_2303_03529_gb300/workload.py.

The paper's E_rep (Sec. III.D) is a pair potential fitted to DFT binding
curves that are not available.  Without any repulsion the synthetic
iron-like cell collapses (its electronic energy falls by about 38 eV per atom
per Angstrom of lattice constant near a = 2.87 A).  The stand-in
Phi(r) = A exp(-b (r - r0)) s(r), b = 3 / A, takes A such that the ideal
4x4x4 bcc cell at a = 2.87 A (n = 0, which is the self-consistent point of
the ideal cell by symmetry) has dU/da = 0, i.e. zero pressure.
"""
from __future__ import annotations

import numpy as np

from . import electronic, energy, model


def _ideal(a, nc):
    R = np.zeros((2 * nc ** 3, 3))
    p_ = 0
    for i in range(nc):
        for j in range(nc):
            for k in range(nc):
                R[p_] = np.array([i, j, k]) * a
                R[p_ + 1] = R[p_] + 0.5 * a
                p_ += 2
    return R, np.full(3, nc * a)


def fit(params, a=2.87, nc=4, h=2e-3):
    def e_el(aa):
        R, cell = _ideal(aa, nc)
        d = electronic.density(R, cell, np.zeros(2 * len(R)), params)
        return energy.shadow_energy(d, model.build_h0(R, cell, params))["U"]

    def e_rep1(aa):
        R, cell = _ideal(aa, nc)
        return model.repulsive_energy(R, cell, params.replace(rep_A=1.0))

    d_el = (e_el(a + h) - e_el(a - h)) / (2 * h)
    d_rep = (e_rep1(a + h) - e_rep1(a - h)) / (2 * h)
    return -d_el / d_rep


if __name__ == "__main__":
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2303_03529_gb300.workload import ModelParams
    print(repr(fit(ModelParams())))
