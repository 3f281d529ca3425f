"""Pins of the paper-general oracle (oracle/general.py): non-orthogonal
basis and l-resolved charges and spins (Sec. III.A, Eqs. D_min, nfromP,
ShadowELatte).

* With S = I and one group per atom it is the orthogonal per-atom oracle,
  itself pinned by tests/test_oracle_*.py (agreement to rounding).
* With the overlap and the shells on: sum_sigma Tr[D S] = N_e, C^T S C = I,
  D S D = D as kT -> 0 on a gapped variant, the response against central
  finite differences of q[n + lambda v], and the forces (with the Pulay and
  Mulliken-overlap terms) against central finite differences of U(R).
* Without hopping and overlap the levels split per shell by 2 J_l s and the
  d-shell spin response has the closed form of the per-atom test.
"""
import numpy as np
import pytest

from oracle import electronic, energy, general, model
from paper_2303_03529_gb300 import workload as wl


@pytest.fixture(scope="module")
def gen16():
    w = wl.fe16_general()
    return w, general.density(w.R, w.cell, w.n0, w.params)


def test_reduces_to_orthogonal_per_atom_oracle():
    w = wl.fe16()
    p = w.params
    d0 = electronic.density(w.R, w.cell, w.n0, p)
    g0 = general.density(w.R, w.cell, w.n0, p)
    assert np.abs(d0.q - g0.q).max() < 1e-12 and abs(d0.mu - g0.mu) < 1e-12
    v = wl.random_direction(w.n_atoms, 3)
    assert np.abs(d0.response(v)[0] - g0.response(v)[0]).max() < 1e-12
    H0 = model.build_h0(w.R, w.cell, p)
    e0, e1 = energy.shadow_energy(d0, H0), general.shadow_energy(g0, H0)
    for k in e0:
        assert abs(e0[k] - e1[k]) < 1e-10, k
    assert np.abs(energy.forces(d0, w.R, w.cell) - general.forces(g0, w.R, w.cell)).max() < 1e-12


def test_overlap_metric_identities(gen16):
    w, d = gen16
    S = d.S
    assert np.allclose(S, S.T, atol=0) and np.allclose(np.diag(S), 1.0)
    assert np.linalg.eigvalsh(S).min() > 0.5
    assert abs(np.abs(S - np.eye(S.shape[0])).max()) > 0.05      # really non-orthogonal
    for c in d.chans:
        np.testing.assert_allclose(c.C.T @ S @ c.C, np.eye(S.shape[0]), atol=1e-11)
    ntot = sum(np.trace(D @ S) for D in d.D)
    assert abs(ntot - d.n_elec) < 1e-10
    assert abs(d.charge.sum()) < 1e-10            # neutral in total
    assert d.q.size == 2 * 3 * w.n_atoms


def test_idempotent_in_overlap_metric_at_low_temperature():
    """10 e/atom fill the d shell and leave s empty (gapped variant with weak
    hopping): as kT -> 0, D S D -> D."""
    w = wl.fe16_general()
    p = w.params.replace(kT=0.02, n_elec_per_atom=10.0, W=0.0, J_l=(0.0, 0.0, 0.0),
                         V0=tuple(0.1 * v for v in w.params.V0))
    d = general.density(w.R, w.cell, np.zeros(6 * w.n_atoms), p)
    for D in d.D:
        assert np.abs(D @ d.S @ D - D).max() < 1e-8


def test_response_against_finite_differences(gen16):
    w, d = gen16
    v = wl.random_direction(3 * w.n_atoms, 17)
    qv, _ = d.response(v)
    lam = 1e-5
    H0 = model.build_h0(w.R, w.cell, w.params)
    G = model.gamma_matrix(w.R, w.cell, w.params)
    qp = general.GDensity(H0, d.S, G, w.n0 + lam * v, w.params, mu_guess=d.mu).q
    qm = general.GDensity(H0, d.S, G, w.n0 - lam * v, w.params, mu_guess=d.mu).q
    fd = (qp - qm) / (2 * lam)
    assert np.abs(qv - fd).max() < 1e-8 * max(1.0, np.abs(fd).max())
    assert np.abs(qv).max() > 1e-3


def _U(R, cell, n, p, mu):
    d = general.density(R, cell, n, p, mu_guess=mu)
    H0 = model.build_h0(R, cell, p)
    return general.shadow_energy(d, H0, model.repulsive_energy(R, cell, p))["U"]


def test_forces_against_finite_differences(gen16):
    """F = -dU/dR at constant n: the Pulay term (energy-weighted D) and the
    overlap inside the Mulliken occupations both enter; either sign wrong
    moves F by ~0.1-1 eV/A here."""
    w, d = gen16
    F = general.forces(d, w.R, w.cell)
    assert np.abs(F.sum(axis=0)).max() < 1e-9           # translation invariance
    rng = np.random.default_rng(4)
    h = 1e-4
    for _ in range(4):
        a, c = int(rng.integers(w.n_atoms)), int(rng.integers(3))
        Rp, Rm = w.R.copy(), w.R.copy()
        Rp[a, c] += h
        Rm[a, c] -= h
        fd = -(_U(Rp, w.cell, w.n0, w.params, d.mu) - _U(Rm, w.cell, w.n0, w.params, d.mu)) / (2 * h)
        assert abs(F[a, c] - fd) < 2e-6, (a, c, F[a, c], fd)


def _atomic_pair(p):
    p0 = p.replace(V0=(0.0,) * 10, S0=(0.0,) * 10)
    R = np.array([[1.0, 1.0, 1.0], [9.0, 8.0, 7.0]])
    cell = np.array([40.0, 40.0, 40.0])
    return p0, model.build_h0(R, cell, p0), general.overlap(R, cell, p0), \
        model.gamma_matrix(R, cell, p0)


def test_shell_resolved_spin_split():
    p0, H0, S, G = _atomic_pair(wl.general_model(wl.ModelParams()))
    # atom 0: s spin 0.2 in its s shell, 0.5 in p, -0.4 in d; atom 1 none
    up = np.array([[0.1, 0.25, -0.2], [0.0, 0.0, 0.0]])
    dn = np.array([[-0.1, -0.25, 0.2], [0.0, 0.0, 0.0]])
    n = np.concatenate([up.reshape(-1), dn.reshape(-1)])
    vu, vd = general.potentials(n, G, p0)
    Hu, Hd = general.hamiltonian(H0, S, vu), general.hamiltonian(H0, S, vd)
    split = (np.diag(Hu) - np.diag(Hd))[:9]
    expect = 2 * np.array([-0.1 * 0.2] + [-0.1 * 0.5] * 3 + [-0.3 * -0.4] * 5)
    np.testing.assert_allclose(split, expect, atol=1e-15)
    np.testing.assert_allclose(np.diag(Hu - Hd)[9:], 0.0, atol=1e-15)


def test_shell_resolved_spin_response_closed_form():
    """No hopping or overlap, n = 0: the d shell holds 4 of 5 electrons per
    spin (f_d = 0.8, mu = -6 + kT ln 4); a d-shell spin direction
    v = delta (e_up,0,d - e_dn,0,d) shifts atom 0's d levels by
    +-2 J_d delta and moves each channel's d occupation by
    -/+ 2 J_d delta beta 5 f_d (1 - f_d) = +-4.8 delta (J_d = -0.3 eV)."""
    p0, H0, S, G = _atomic_pair(wl.general_model(wl.ModelParams()))
    d = general.GDensity(H0, S, G, np.zeros(12), p0)
    assert abs(d.mu - (-6.0 + 0.1 * np.log(4.0))) < 1e-12
    delta = 0.01
    v = np.zeros(12)
    v[2], v[6 + 2] = delta, -delta
    qv, dmu = d.response(v)
    expect = np.zeros(12)
    expect[2], expect[8] = 4.8 * delta, -4.8 * delta
    assert abs(dmu) < 1e-14
    np.testing.assert_allclose(qv, expect, atol=1e-12)
