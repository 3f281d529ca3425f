"""Oracle: the paper-general form of the SCC tight-binding model, with a
non-orthogonal basis and l-resolved charges and spins (Sec. III.A).

Test infrastructure only (see oracle/__init__.py).

* Overlap S (Sec. II.C): S_ii = 1 on site, and between atoms the
  Slater-Koster blocks of overlap integrals S0_b exp(-s_decay (r - r0)) s(r),
  the same two-center table as H0 (model.sk_block) with the overlap
  integrals in place of the hopping ones.
* Eq. D_min with the congruence transform: D = Z f(Z^T H Z) Z^T for any Z
  with Z^T S Z = I.  Written here by its definition, the generalized
  eigenproblem H c = eps S c with C^T S C = I (scipy.linalg.eigh(H, S)):
  D = C diag(f(eps - mu)) C^T, one mu for both spins with
  sum_sigma Tr[D S] = N_e (Eq. directBO's constraint).
* Mulliken occupations with S (Eq. nfromP and the q_I, m_l equations):
  n^sigma_{I,g} = sum_{i in (I, g)} sum_j (D - D0)_ij S_ji, with g the atom's
  shell l of orbital i when l_resolved, else one group per atom.  The
  extended vector is n = [n_up (N_at x G); n_dn (N_at x G)], G = 3 or 1.
* Hamiltonian: the derivative of the shadow energy (Eq. ShadowELatte) with
  respect to D^sigma, with the occupations written through S:
  H^sigma = H0 + 1/2 S o (v^sigma 1^T + 1 v^sigma^T), where the orbital
  potential is v^sigma_i = (gamma n_tot)_I + sigma J_g s_{I,g} for i in
  (I, g), n_tot the atom totals and s = n_up - n_dn per group.
  J_g = J_l[g] (l-dependent Stoner parameters, Sec. III.A) when l_resolved,
  else W / 2 for the single per-atom group.
* Shadow energy: E_band = sum_sigma Tr[H0 (D - D0)],
  E_coul = 1/2 sum (2 q - n) gamma n over atom totals,
  E_spin = 1/2 sum_I sum_g (2 m_{I,g} - s_{I,g}) J_g s_{I,g} (the double sum
  over l, l' printed with a single-index J is read as a single sum),
  E_ent of the orthogonalized D (Eq. Entropy, eigenvalue form).
* Forces at constant n, D stationary: per bond (K, J, d = R_J - R_K)
  F_K += 2 sum_ab [D_ab dE0_ab/dd + (Dv_ab - W_ab) dS_ab/dd] with
  Dv_ab = sum_sigma D^sigma_ab (v^sigma_a + v^sigma_b) / 2 (the S inside the
  Mulliken occupations) and the energy-weighted W = sum_sigma C diag(f eps) C^T
  (the normalization C^T S C = I), plus the Coulomb and repulsion terms of
  energy.forces.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import electronic, model

NORB = model.NORB
SHELL = model.ELL          # s -> 0, p -> 1, d -> 2
CSTEP = 1e-30


class _Params:
    """Parameter view with the overlap integrals in place of the hopping ones
    and on-site values 1, so that model.build_h0 / sk_block build S."""

    def __init__(self, p):
        for f in ("r0", "r_cut", "r_on"):
            setattr(self, f, getattr(p, f))
        self.V0 = tuple(p.S0)
        self.q_decay = p.s_decay
        self.eps_s = self.eps_p = self.eps_d = 1.0


def overlap(R, cell, p):
    """Dense S (9 N_at square): identity on site plus the image-summed
    Slater-Koster overlap blocks."""
    return model.build_h0(R, cell, _Params(p))


def overlap_block(d, p):
    return model.sk_block(d, _Params(p))


def n_groups(p):
    return 3 if p.l_resolved else 1


def orbital_group(p):
    return SHELL.copy() if p.l_resolved else np.zeros(NORB, dtype=int)


def stoner(p):
    """J_g per group: the l-dependent Stoner parameters, or W / 2 per atom."""
    return np.array(p.J_l, dtype=np.float64) if p.l_resolved else np.array([0.5 * p.W])


def potentials(n, gamma, p):
    """Orbital potentials (v_up, v_dn), each 9 N_at, for the extended vector
    n (or a direction: the map is linear)."""
    nat = gamma.shape[0]
    G = n_groups(p)
    nu = np.asarray(n[:nat * G]).reshape(nat, G)
    nd = np.asarray(n[nat * G:]).reshape(nat, G)
    coul = gamma @ (nu + nd).sum(axis=1)
    s = nu - nd
    J = stoner(p)
    grp = orbital_group(p)
    vu = coul[:, None] + (J[None, :] * s)[:, grp]
    vd = coul[:, None] - (J[None, :] * s)[:, grp]
    return vu.reshape(-1), vd.reshape(-1)


def hamiltonian(H0, S, v):
    """H0 + 1/2 S o (v 1^T + 1 v^T)."""
    return H0 + 0.5 * S * (v[:, None] + v[None, :])


def group_sums(x, p, nat):
    """Sum of a per-orbital vector over the orbitals of each (atom, group)."""
    G = n_groups(p)
    grp = orbital_group(p)
    out = np.zeros((nat, G))
    xr = np.asarray(x).reshape(nat, NORB)
    for a in range(NORB):
        out[:, grp[a]] += xr[:, a]
    return out.reshape(-1)


class GeneralChannel:
    """Generalized eigendecomposition H c = eps S c, C^T S C = I."""

    def __init__(self, H, S):
        self.eps, self.C = scipy.linalg.eigh(H, S)


class GDensity:
    """D_up, D_dn, mu and the S-weighted occupations q (2 N_at G) for given
    H0, S, gamma and n."""

    def __init__(self, H0, S, gamma, n, p, mu_guess=None):
        self.p = p
        self.beta = 1.0 / p.kT
        self.S = S
        self.gamma = gamma
        self.nat = gamma.shape[0]
        self.G = n_groups(p)
        self.n = np.asarray(n, dtype=np.float64).copy()
        self.v = potentials(self.n, gamma, p)
        self.H = tuple(hamiltonian(H0, S, v) for v in self.v)
        self.chans = tuple(GeneralChannel(H, S) for H in self.H)
        self.n_elec = p.n_elec_per_atom * self.nat
        self.mu = electronic.find_mu(self.chans, self.n_elec, self.beta, mu_guess=mu_guess)
        self.occ = tuple(electronic.fermi(c.eps - self.mu, self.beta) for c in self.chans)
        self.occ_c = tuple(electronic.fermi(self.mu - c.eps, self.beta) for c in self.chans)
        self.D = tuple((c.C * f) @ c.C.T for c, f in zip(self.chans, self.occ))
        self.W = tuple((c.C * (f * c.eps)) @ c.C.T for c, f in zip(self.chans, self.occ))
        d0 = np.tile(model.d0_diag(p), self.nat)
        self.q_spin = tuple(group_sums(np.einsum("ij,ji->i", D, S) - d0, p, self.nat)
                            for D in self.D)

    @property
    def q(self):
        return np.concatenate(self.q_spin)

    @property
    def charge(self):
        """Atom totals q_I (both spins, all groups)."""
        return (self.q_spin[0] + self.q_spin[1]).reshape(self.nat, self.G).sum(axis=1)

    @property
    def spin(self):
        """Spin moments per (atom, group)."""
        return self.q_spin[0] - self.q_spin[1]

    def residual(self):
        return self.q - self.n

    def response(self, v):
        """q_v = d q[n + lambda v]/d lambda (Eq. fv) by perturbation theory in
        the generalized eigenbasis: dH^sigma = 1/2 S o (dv 1^T + 1 dv^T),
        dH' = C^T dH C, dD = C (F o (dH' - dmu I)) C^T with the divided
        differences F and the common dmu from sum_sigma Tr[dD S] = 0."""
        v = np.asarray(v, dtype=np.float64)
        dv = potentials(v, self.gamma, self.p)
        if not hasattr(self, "_F"):
            self._F = tuple(electronic.fermi_divided_differences(c.eps, self.mu, self.beta)
                            for c in self.chans)
        dHs = [c.C.T @ hamiltonian(np.zeros_like(self.S), self.S, x) @ c.C
               for c, x in zip(self.chans, dv)]
        num = sum(float(np.sum(np.diag(F) * np.diag(dH))) for F, dH in zip(self._F, dHs))
        den = sum(float(np.sum(np.diag(F))) for F in self._F)
        dmu = num / den
        qv = []
        for c, F, dH in zip(self.chans, self._F, dHs):
            dD = c.C @ (F * (dH - dmu * np.eye(dH.shape[0]))) @ c.C.T
            qv.append(group_sums(np.einsum("ij,ji->i", dD, self.S), self.p, self.nat))
        return np.concatenate(qv), dmu

    def fv(self, v):
        return self.response(v)[0] - np.asarray(v)

    def entropy_term(self):
        tot = 0.0
        for f, g in zip(self.occ, self.occ_c):
            with np.errstate(divide="ignore", invalid="ignore"):
                a = np.where(f > 0, f * np.log(f), 0.0)
                b = np.where(g > 0, g * np.log(g), 0.0)
            tot += float(np.sum(a + b))
        return self.p.kT * tot


def density(R, cell, n, p, mu_guess=None):
    H0 = model.build_h0(R, cell, p)
    S = overlap(R, cell, p)
    G = model.gamma_matrix(R, cell, p)
    return GDensity(H0, S, G, n, p, mu_guess=mu_guess)


def shadow_energy(dens, H0, e_rep=0.0):
    """U and its parts (Eq. ShadowELatte at the stationary D)."""
    p = dens.p
    nat, G = dens.nat, dens.G
    d0 = np.tile(model.d0_diag(p), nat)
    e_band = sum(float(np.sum(H0 * (D - np.diag(d0)))) for D in dens.D)
    n = dens.n
    nu, nd = n[:nat * G].reshape(nat, G), n[nat * G:].reshape(nat, G)
    n_tot = (nu + nd).sum(axis=1)
    s = (nu - nd).reshape(-1)
    e_coul = 0.5 * float((2 * dens.charge - n_tot) @ dens.gamma @ n_tot)
    J = np.tile(stoner(p), nat)
    e_spin = 0.5 * float(np.sum((2 * dens.spin - s) * J * s))
    e_ent = dens.entropy_term()
    U = e_band + e_coul + e_spin + e_ent + e_rep
    return dict(U=U, band=e_band, coul=e_coul, spin=e_spin, entropy=e_ent, rep=e_rep)


def _block_gradient(block_fn, d, p):
    out = np.empty((3, NORB, NORB))
    for c in range(3):
        dc = np.array(d, dtype=np.complex128)
        dc[c] += 1j * CSTEP
        out[c] = np.imag(block_fn(dc, p)) / CSTEP
    return out


def forces(dens, R, cell):
    """F (N_at x 3, eV/Angstrom) at constant n (complex-step block
    derivatives; Coulomb and repulsion terms as in energy.forces)."""
    p = dens.p
    nat = dens.nat
    R = np.asarray(R, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    F = np.zeros((nat, 3))
    Dsum = dens.D[0] + dens.D[1]
    Wsum = dens.W[0] + dens.W[1]
    Dv = sum(0.5 * D * (v[:, None] + v[None, :]) for D, v in zip(dens.D, dens.v))
    for K, J, d in model.image_bonds(R, cell, p.r_cut):
        if K == J:
            continue
        sl = (slice(NORB * K, NORB * K + NORB), slice(NORB * J, NORB * J + NORB))
        gH = _block_gradient(model.sk_block, d, p)
        gS = _block_gradient(overlap_block, d, p)
        F[K] += 2.0 * np.einsum("ab,cab->c", Dsum[sl], gH)
        F[K] += 2.0 * np.einsum("ab,cab->c", Dv[sl] - Wsum[sl], gS)
        for c in range(3):
            dc = np.array(d, dtype=np.complex128)
            dc[c] += 1j * CSTEP
            F[K, c] += np.imag(model.pair_repulsion(np.sqrt(dc @ dc), p)) / CSTEP
    G = dens.G
    n = dens.n
    b = (n[:nat * G] + n[nat * G:]).reshape(nat, G).sum(axis=1)
    a = 2.0 * dens.charge - b
    dd = R[None, :, :] - R[:, None, :]
    dd = dd - cell * np.round(dd / cell)
    gg = np.empty((nat, nat, 3))
    for c in range(3):
        dc = dd.astype(np.complex128)
        dc[:, :, c] += 1j * CSTEP
        val = p.coulomb_k / np.sqrt(np.sum(dc * dc, axis=2) + (p.coulomb_k / p.U) ** 2)
        gg[:, :, c] = np.imag(val) / CSTEP
    Wm = 0.5 * a[:, None] * b[None, :]
    np.fill_diagonal(Wm, 0.0)
    F -= np.einsum("ij,ijc->jc", Wm, gg)
    F += np.einsum("ij,ijc->ic", Wm, gg)
    return F
