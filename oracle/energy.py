"""Oracle: shadow potential energy U(R, n) and forces -dU/dR at constant n.

Test infrastructure only (see oracle/__init__.py).

Eq. ShadowELatte evaluated at the stationary D of Eq. ShadowULatte, per atom
(no l resolution), orthogonal basis:
  E_band = sum_sigma Tr[H0 (D^sigma - D0^sigma)]
  E_coul = 1/2 sum_IJ (2 q_I - n_I) gamma_IJ n_J
  E_spin = 1/2 sum_I (2 m_I - s_I) J s_I with J = W/2, i.e. (W/4) sum (2m - s) s
  E_ent  = kT sum_sigma sum_a [f ln f + (1 - f) ln(1 - f)]   (Eq. Entropy)
  U      = E_band + E_coul + E_spin + E_ent + E_rep,
  E_rep  = 1/2 sum_{i != j} Phi(R_ij)  (Sec. III.D, Phi from model.pair_repulsion).
Forces (Eq. EqMot, first line): because D is stationary, only the explicit
R-dependence of H0 and gamma enters:
  F_K = -sum_sigma Tr[D^sigma dH0/dR_K] - 1/2 sum_IJ (2q_I - n_I) n_J dgamma_IJ/dR_K.
The derivatives of the Slater-Koster blocks and of gamma are complex-step
derivatives of model.sk_block and of the gamma formula (exact to rounding).
"""
from __future__ import annotations

import numpy as np

from . import model

NORB = model.NORB
CSTEP = 1e-30


def shadow_energy(dens, H0, e_rep=0.0):
    """Returns dict with U and its parts for an electronic.Density; e_rep is
    model.repulsive_energy(R, cell, p), passed in because it needs R."""
    p = dens.p
    d0 = np.tile(model.d0_diag(p), dens.nat)
    e_band = 0.0
    for D in dens.D:
        e_band += float(np.sum(H0 * (D - np.diag(d0))))
    nat = dens.nat
    n = dens.n
    n_tot = n[:nat] + n[nat:]
    s = n[:nat] - n[nat:]
    q = dens.charge
    m = dens.spin
    e_coul = 0.5 * float((2 * q - n_tot) @ dens.gamma @ n_tot)
    e_spin = 0.25 * p.W * float(np.sum((2 * m - s) * s))
    e_ent = dens.entropy_term()
    U = e_band + e_coul + e_spin + e_ent + e_rep
    return dict(U=U, band=e_band, coul=e_coul, spin=e_spin, entropy=e_ent, rep=e_rep)


def sk_gradient(d, p):
    """dE_ab/dd_x, dE_ab/dd_y, dE_ab/dd_z (3 x 9 x 9) by the complex step."""
    out = np.empty((3, NORB, NORB))
    for c in range(3):
        dc = np.array(d, dtype=np.complex128)
        dc[c] += 1j * CSTEP
        out[c] = np.imag(model.sk_block(dc, p)) / CSTEP
    return out


def forces(dens, R, cell):
    """F (N_at x 3, eV/Angstrom) at constant n."""
    p = dens.p
    nat = dens.nat
    R = np.asarray(R, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    F = np.zeros((nat, 3))
    Dsum = dens.D[0] + dens.D[1]
    # band term: F_K = 2 sum_{bonds (K, J, d), J != K} sum_ab D_{Ka,Jb} dE_ab/dd
    for K, J, d in model.image_bonds(R, cell, p.r_cut):
        if K == J:
            continue  # a self-image bond does not depend on R_K
        blk = Dsum[NORB * K:NORB * K + NORB, NORB * J:NORB * J + NORB]
        g = sk_gradient(d, p)
        F[K] += 2.0 * np.einsum("ab,cab->c", blk, g)
        # repulsion: E_rep = 1/2 sum_bonds Phi(|d|); each pair enters as (K, J)
        # and (J, K), so F_K = sum_{bonds (K, J, d)} dPhi(|d|)/dd
        for c in range(3):
            dc = np.array(d, dtype=np.complex128)
            dc[c] += 1j * CSTEP
            F[K, c] += np.imag(model.pair_repulsion(np.sqrt(dc @ dc), p)) / CSTEP
    # Coulomb term with a = 2q - n, b = n (per-atom totals):
    # E_coul = 1/2 sum_IJ a_I gamma_IJ(d_IJ) b_J, d_IJ = minimum image of R_J - R_I
    n = dens.n
    b = n[:nat] + n[nat:]
    a = 2.0 * dens.charge - b
    d = R[None, :, :] - R[:, None, :]
    d = d - cell * np.round(d / cell)
    gg = np.empty((nat, nat, 3))
    for c in range(3):
        dc = d.astype(np.complex128)
        dc[:, :, c] += 1j * CSTEP
        val = p.coulomb_k / np.sqrt(np.sum(dc * dc, axis=2) + (p.coulomb_k / p.U) ** 2)
        gg[:, :, c] = np.imag(val) / CSTEP
    Wm = 0.5 * a[:, None] * b[None, :]
    np.fill_diagonal(Wm, 0.0)
    # d gamma_IJ / d R_J = +gg[I, J], d gamma_IJ / d R_I = -gg[I, J]
    F -= np.einsum("ij,ijc->jc", Wm, gg)
    F += np.einsum("ij,ijc->ic", Wm, gg)
    return F
