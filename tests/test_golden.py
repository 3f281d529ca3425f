"""The oracle against its stored values for the 16-atom cell
(tests/golden/fe16_fp64.json, written by tests/golden/make_golden.py from
the oracle alone; the paper prints no worked example).  A regression guard:
any change to the oracle's arithmetic shows here first, and the commit that
makes it must say which passage of the paper justifies it."""
import json
import os

import numpy as np

from oracle import dynamics, electronic, energy, model
from paper_2303_03529_gb300 import workload as wl

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fe16_fp64.json")


def test_oracle_reproduces_golden_fe16():
    g = json.load(open(GOLD))
    w = wl.fe16()
    d = electronic.density(w.R, w.cell, w.n0, w.params)
    assert abs(d.mu - g["mu"]) < 1e-12
    np.testing.assert_allclose(d.q, g["q"], atol=1e-12)
    np.testing.assert_allclose(d.spin, g["spin"], atol=1e-12)
    qv, dmu = d.response(wl.random_direction(w.n_atoms, g["response_direction_seed"]))
    np.testing.assert_allclose(qv, g["qv"], atol=1e-12)
    assert abs(dmu - g["dmu"]) < 1e-12
    e = energy.shadow_energy(d, model.build_h0(w.R, w.cell, w.params),
                             model.repulsive_energy(w.R, w.cell, w.params))
    for k, v in g["energies"].items():
        assert abs(e[k] - v) < 1e-10, k
    np.testing.assert_allclose(energy.forces(d, w.R, w.cell), g["forces"], atol=1e-11)


def test_oracle_scf_reproduces_golden_fixed_point():
    g = json.load(open(GOLD))
    w = wl.fe16()
    res = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-10)
    assert res["iters"] == g["scf_iters"]
    np.testing.assert_allclose(res["n"], g["scf_n"], atol=1e-11)
    assert abs(res["mu"] - g["scf_mu"]) < 1e-11
