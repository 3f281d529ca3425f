"""Oracle: the SCC tight-binding model of Sec. III.A (Eq. ELatte).

Test infrastructure only (see oracle/__init__.py).

* H0: charge-independent Slater-Koster Hamiltonian in an orthogonal s, p, d
  basis (Sec. III.A: "charge-independent Slater-Koster tight-binding
  Hamiltonian"; orthogonal basis, so S = I and Z = I in Eq. D_min).  The
  two-center integrals are the Slater-Koster (1954) table in direction cosines
  (l, m, n) of d = R_J - R_I, written out below entry by entry.  Periodic
  images: all images with |d| < r_cut are summed (Gamma-point Hamiltonian).
* gamma: screened Coulomb matrix, gamma_II = U and gamma_IJ -> k/r at large r
  (Sec. III.A text after Eq. ELatte), minimum-image distance.
* H_sigma[n]: derivative of the linearized shadow energy (Eq. ShadowELatte)
  with respect to D^sigma: H0 + diag((gamma n)_I + sigma (W/2) s_I) on every
  orbital of atom I, with n_I = n_up + n_dn and s_I = n_up - n_dn.

Orbital order per atom: s, px, py, pz, dxy, dyz, dzx, dx2-y2, d3z2-r2.
All functions accept complex displacements so that forces can be taken by the
complex-step derivative (an exact first derivative, no subtraction).
"""
from __future__ import annotations

import numpy as np

NORB = 9
ELL = np.array([0, 1, 1, 1, 2, 2, 2, 2, 2])
S3 = np.sqrt(3.0)


def switch(r, r_on, r_cut):
    """C2 quintic switch: 1 below r_on, 1 - 10x^3 + 15x^4 - 6x^5 on
    [r_on, r_cut] with x = (r - r_on)/(r_cut - r_on), 0 beyond.
    Branches are taken on the real part so complex steps pass through."""
    rr = np.real(r)
    if rr <= r_on:
        return 1.0 + 0.0 * r
    if rr >= r_cut:
        return 0.0 * r
    x = (r - r_on) / (r_cut - r_on)
    return 1.0 - 10.0 * x ** 3 + 15.0 * x ** 4 - 6.0 * x ** 5


def bond_integrals(r, p):
    """The ten bond integrals V_b(r) = V0_b exp(-q (r - r0)) s(r)."""
    rad = np.exp(-p.q_decay * (r - p.r0)) * switch(r, p.r_on, p.r_cut)
    return [v0 * rad for v0 in p.V0]


def sk_block(d, p):
    """9x9 two-center block E[a, b] = <phi_a(0)|H|phi_b(d)> for displacement d.

    Entries for a <= b are the Slater-Koster table; entries for a > b follow
    from E_ba(d) = E_ab(-d) = (-1)^(l_a + l_b) E_ab(d)."""
    d = np.asarray(d)
    r = np.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
    l, m, n = d[0] / r, d[1] / r, d[2] / r
    sss, sps, sds, pps, ppp, pds, pdp, dds, ddp, ddd = bond_integrals(r, p)
    l2, m2, n2 = l * l, m * m, n * n
    lm2 = l2 - m2           # l^2 - m^2
    z2f = n2 - 0.5 * (l2 + m2)  # n^2 - (l^2 + m^2)/2

    E = np.zeros((NORB, NORB), dtype=np.result_type(d.dtype, np.float64))
    s, x, y, z, xy, yz, zx, x2, z2 = range(9)
    # s-s, s-p, s-d
    E[s, s] = sss
    E[s, x] = l * sps
    E[s, y] = m * sps
    E[s, z] = n * sps
    E[s, xy] = S3 * l * m * sds
    E[s, yz] = S3 * m * n * sds
    E[s, zx] = S3 * n * l * sds
    E[s, x2] = 0.5 * S3 * lm2 * sds
    E[s, z2] = z2f * sds
    # p-p
    E[x, x] = l2 * pps + (1 - l2) * ppp
    E[y, y] = m2 * pps + (1 - m2) * ppp
    E[z, z] = n2 * pps + (1 - n2) * ppp
    E[x, y] = l * m * (pps - ppp)
    E[x, z] = l * n * (pps - ppp)
    E[y, z] = m * n * (pps - ppp)
    # p-d
    E[x, xy] = S3 * l2 * m * pds + m * (1 - 2 * l2) * pdp
    E[x, yz] = S3 * l * m * n * pds - 2 * l * m * n * pdp
    E[x, zx] = S3 * l2 * n * pds + n * (1 - 2 * l2) * pdp
    E[y, xy] = S3 * m2 * l * pds + l * (1 - 2 * m2) * pdp
    E[y, yz] = S3 * m2 * n * pds + n * (1 - 2 * m2) * pdp
    E[y, zx] = S3 * l * m * n * pds - 2 * l * m * n * pdp
    E[z, xy] = S3 * l * m * n * pds - 2 * l * m * n * pdp
    E[z, yz] = S3 * n2 * m * pds + m * (1 - 2 * n2) * pdp
    E[z, zx] = S3 * n2 * l * pds + l * (1 - 2 * n2) * pdp
    E[x, x2] = 0.5 * S3 * l * lm2 * pds + l * (1 - lm2) * pdp
    E[y, x2] = 0.5 * S3 * m * lm2 * pds - m * (1 + lm2) * pdp
    E[z, x2] = 0.5 * S3 * n * lm2 * pds - n * lm2 * pdp
    E[x, z2] = l * z2f * pds - S3 * l * n2 * pdp
    E[y, z2] = m * z2f * pds - S3 * m * n2 * pdp
    E[z, z2] = n * z2f * pds + S3 * n * (l2 + m2) * pdp
    # d-d
    E[xy, xy] = 3 * l2 * m2 * dds + (l2 + m2 - 4 * l2 * m2) * ddp + (n2 + l2 * m2) * ddd
    E[yz, yz] = 3 * m2 * n2 * dds + (m2 + n2 - 4 * m2 * n2) * ddp + (l2 + m2 * n2) * ddd
    E[zx, zx] = 3 * n2 * l2 * dds + (n2 + l2 - 4 * n2 * l2) * ddp + (m2 + n2 * l2) * ddd
    E[xy, yz] = 3 * l * m2 * n * dds + l * n * (1 - 4 * m2) * ddp + l * n * (m2 - 1) * ddd
    E[xy, zx] = 3 * l2 * m * n * dds + m * n * (1 - 4 * l2) * ddp + m * n * (l2 - 1) * ddd
    E[yz, zx] = 3 * l * m * n2 * dds + l * m * (1 - 4 * n2) * ddp + l * m * (n2 - 1) * ddd
    E[xy, x2] = 1.5 * l * m * lm2 * dds - 2 * l * m * lm2 * ddp + 0.5 * l * m * lm2 * ddd
    E[yz, x2] = 1.5 * m * n * lm2 * dds - m * n * (1 + 2 * lm2) * ddp + m * n * (1 + 0.5 * lm2) * ddd
    E[zx, x2] = 1.5 * n * l * lm2 * dds + n * l * (1 - 2 * lm2) * ddp - n * l * (1 - 0.5 * lm2) * ddd
    E[xy, z2] = S3 * l * m * z2f * dds - 2 * S3 * l * m * n2 * ddp + 0.5 * S3 * l * m * (1 + n2) * ddd
    E[yz, z2] = S3 * m * n * z2f * dds + S3 * m * n * (l2 + m2 - n2) * ddp - 0.5 * S3 * m * n * (l2 + m2) * ddd
    E[zx, z2] = S3 * l * n * z2f * dds + S3 * l * n * (l2 + m2 - n2) * ddp - 0.5 * S3 * l * n * (l2 + m2) * ddd
    E[x2, x2] = 0.75 * lm2 ** 2 * dds + (l2 + m2 - lm2 ** 2) * ddp + (n2 + 0.25 * lm2 ** 2) * ddd
    E[x2, z2] = 0.5 * S3 * lm2 * z2f * dds + S3 * n2 * (m2 - l2) * ddp + 0.25 * S3 * (1 + n2) * lm2 * ddd
    E[z2, z2] = z2f ** 2 * dds + 3 * n2 * (l2 + m2) * ddp + 0.75 * (l2 + m2) ** 2 * ddd
    # lower triangle by inversion parity
    for a in range(NORB):
        for b in range(a):
            E[a, b] = (-1.0) ** (ELL[a] + ELL[b]) * E[b, a]
    return E


def pair_repulsion(r, p):
    """Phi(r) = A exp(-b (r - r0)) s(r), the pair term of
    E_rep = 1/2 sum_{i != j} Phi(R_ij) (Sec. III.D).  The paper's Phi was
    fitted to DFT binding curves that are not available; here A is fitted
    (oracle/fit_repulsion.py) so that the ideal 4x4x4 bcc cell at a = 2.87 A
    is at zero pressure."""
    return p.rep_A * np.exp(-p.rep_b * (r - p.r0)) * switch(r, p.r_on, p.r_cut)


def repulsive_energy(R, cell, p):
    """E_rep = 1/2 sum over image bonds (each unordered pair appears twice)."""
    tot = 0.0
    for _, _, d in image_bonds(R, cell, p.r_cut):
        tot += 0.5 * float(pair_repulsion(np.sqrt(d @ d), p))
    return tot


def onsite(p):
    """On-site energies eps_s, eps_p (x3), eps_d (x5)."""
    return np.array([p.eps_s] + [p.eps_p] * 3 + [p.eps_d] * 5)


def d0_diag(p):
    """Neutral-atom occupations per spin and orbital (diagonal of D0^sigma)."""
    return np.array([p.d0_s] + [p.d0_p] * 3 + [p.d0_d] * 5)


def image_bonds(R, cell, r_cut):
    """Every (I, J, d) with d = R_J - R_I + image shift and 0 < |d| < r_cut.

    d is first reduced to the minimum image, then the 27 neighbouring image
    shifts are tried; that covers every image within r_cut whenever
    1.5 * L > r_cut for each box length L."""
    R = np.asarray(R, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    assert np.all(1.5 * cell > r_cut), "cell too small for the 27-image search"
    nat = R.shape[0]
    d = R[None, :, :] - R[:, None, :]
    d = d - cell * np.round(d / cell)
    bonds = []
    shifts = [np.array([i, j, k], dtype=np.float64) * cell
              for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]
    for sh in shifts:
        ds = d + sh
        r = np.sqrt(np.sum(ds * ds, axis=2))
        I, J = np.nonzero((r < r_cut) & (r > 1e-8))
        for a, b in zip(I, J):
            bonds.append((a, b, ds[a, b].copy()))
    assert nat >= 1
    return bonds


def build_h0(R, cell, p):
    """Dense H0 (9 N_at square, float64): on-site energies plus the sum over
    image bonds of the Slater-Koster blocks."""
    nat = R.shape[0]
    H = np.zeros((NORB * nat, NORB * nat))
    eps = onsite(p)
    for I in range(nat):
        H[NORB * I:NORB * I + NORB, NORB * I:NORB * I + NORB] += np.diag(eps)
    for I, J, d in image_bonds(R, cell, p.r_cut):
        H[NORB * I:NORB * I + NORB, NORB * J:NORB * J + NORB] += sk_block(d, p)
    return H


def min_image(d, cell):
    return d - cell * np.round(np.real(d) / cell)


def gamma_matrix(R, cell, p):
    """gamma_IJ = k / sqrt(r_IJ^2 + (k/U)^2), minimum image; gamma_II = U."""
    R = np.asarray(R, dtype=np.float64)
    d = R[None, :, :] - R[:, None, :]
    d = d - cell * np.round(d / cell)
    r2 = np.sum(d * d, axis=2)
    G = p.coulomb_k / np.sqrt(r2 + (p.coulomb_k / p.U) ** 2)
    np.fill_diagonal(G, p.U)
    return G


def spin_potentials(n, gamma, p):
    """Per-atom diagonal shifts (h_up, h_dn) from n = [n_up; n_dn]:
    h_sigma,I = (gamma (n_up + n_dn))_I + sigma (W/2) (n_up - n_dn)_I."""
    nat = gamma.shape[0]
    nu, nd = n[:nat], n[nat:]
    coul = gamma @ (nu + nd)
    s = nu - nd
    return coul + 0.5 * p.W * s, coul - 0.5 * p.W * s


def hamiltonians(H0, n, gamma, p):
    """H_up, H_dn = H0 + diag(h_sigma expanded over the 9 orbitals of each atom)."""
    hu, hd = spin_potentials(n, gamma, p)
    Hu = H0 + np.diag(np.repeat(hu, NORB))
    Hd = H0 + np.diag(np.repeat(hd, NORB))
    return Hu, Hd
