"""Pins of the oracle's density matrix, chemical potential, Mulliken charges
and first-order response (Eqs. D_min, fv, RegJacobian)."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import electronic, model
from paper_2303_03529_gb300 import workload as wl


@pytest.fixture(scope="module")
def dens16():
    w = wl.fe16()
    return w, electronic.density(w.R, w.cell, w.n0, w.params)


def test_trace_symmetry_and_occupation_identities(dens16):
    w, d = dens16
    tot = sum(np.trace(D) for D in d.D)
    assert abs(tot - w.params.n_elec_per_atom * w.n_atoms) < 1e-11
    for D, f in zip(d.D, d.occ):
        np.testing.assert_allclose(D, D.T, atol=1e-14)
        # Tr[D (I - D)] = sum f (1 - f)
        assert abs(np.trace(D) - np.sum(D * D) - np.sum(f * (1 - f))) < 1e-11
    assert abs(np.sum(d.charge)) < 1e-11   # neutral cell


def test_closed_form_no_hopping():
    """All V0 = 0: H is diagonal, D_ii = f(H_ii - mu), and mu solves a scalar
    equation solved here independently with brentq."""
    p = wl.ModelParams(V0=(0.0,) * 10)
    w = wl.make_cell(2, seed=5, params=p)
    rng = np.random.default_rng(1)
    n = np.concatenate([rng.uniform(-0.3, 0.3, 16), rng.uniform(-0.3, 0.3, 16)])
    d = electronic.density(w.R, w.cell, n, p)
    G = model.gamma_matrix(w.R, w.cell, p)
    nu, nd = n[:16], n[16:]
    levels = []
    for sgn in (1, -1):
        shift = G @ (nu + nd) + sgn * 0.5 * p.W * (nu - nd)
        levels.append(np.add.outer(shift, model.onsite(p)))   # (atom, orbital)
    beta = 1.0 / p.kT
    fd = lambda x: 0.5 * (1.0 - np.tanh(0.5 * beta * x))
    count = lambda mu: sum(np.sum(fd(L - mu)) for L in levels) - 8.0 * 16
    mu = brentq(count, -30, 30, xtol=1e-15, rtol=1e-15)
    assert abs(mu - d.mu) < 1e-10
    for s, L in enumerate(levels):
        q_expect = (fd(L - mu) - model.d0_diag(p)).sum(axis=1)
        np.testing.assert_allclose(d.q_spin[s], q_expect, atol=1e-12)


def test_idempotency_low_temperature_gapped():
    """Gapped variant (W = 0, hopping x0.1, 10 electrons/atom): D^2 -> D as kT -> 0."""
    base = wl.ModelParams()
    errs = []
    for kT in (0.1, 0.03, 0.01):   # gap 0.76 eV between -5.69 and -4.93 eV
        p = base.replace(V0=tuple(0.1 * v for v in base.V0), W=0.0,
                         n_elec_per_atom=10.0, kT=kT)
        w = wl.make_cell(2, seed=9, params=p)
        d = electronic.density(w.R, w.cell, np.zeros(32), p)
        errs.append(max(np.abs(D @ D - D).max() for D in d.D))
    assert errs[-1] < 1e-11
    assert errs[0] > errs[1] > errs[2]


def test_divided_differences_match_definition():
    rng = np.random.default_rng(3)
    eps = np.sort(rng.uniform(-3, 3, 40))
    eps[5] = eps[4] + 1e-9     # a near-degenerate pair
    mu, beta = 0.2, 10.0
    F = electronic.fermi_divided_differences(eps, mu, beta)
    f = electronic.fermi(eps - mu, beta)
    for a in range(40):
        for b in range(40):
            if abs(eps[a] - eps[b]) > 1e-3:
                ref = (f[a] - f[b]) / (eps[a] - eps[b])
                assert abs(F[a, b] - ref) < 1e-12 * max(1.0, abs(ref)) + 1e-13
    fc = electronic.fermi(mu - eps, beta)   # 1 - f without cancellation
    np.testing.assert_allclose(np.diag(F), -beta * f * fc, rtol=1e-12, atol=1e-300)
    assert abs(F[4, 5] - (-beta * f[4] * (1 - f[4]))) < 1e-7


def test_response_matches_central_difference(dens16):
    w, d = dens16
    H0 = model.build_h0(w.R, w.cell, w.params)
    G = d.gamma
    for seed in (1, 2):
        v = wl.random_direction(16, seed)
        qv, _ = d.response(v)
        lam = 1e-5
        qp = electronic.Density(H0, G, w.n0 + lam * v, w.params).q
        qm = electronic.Density(H0, G, w.n0 - lam * v, w.params).q
        fd = (qp - qm) / (2 * lam)
        np.testing.assert_allclose(qv, fd, atol=2e-8)
        assert abs(np.sum(qv)) < 1e-11   # common mu keeps the electron count


def test_jacobian_columns_and_spin_swap(dens16):
    w, d = dens16
    J = d.jacobian()
    v = wl.random_direction(16, 5)
    np.testing.assert_allclose(J @ v, d.fv(v), atol=1e-12)
    # swapping the spin channels of n swaps q_up and q_dn
    n_sw = np.concatenate([w.n0[16:], w.n0[:16]])
    d2 = electronic.density(w.R, w.cell, n_sw, w.params)
    np.testing.assert_allclose(d2.q_spin[0], d.q_spin[1], atol=1e-12)
    np.testing.assert_allclose(d2.q_spin[1], d.q_spin[0], atol=1e-12)
    assert abs(d2.mu - d.mu) < 1e-12
