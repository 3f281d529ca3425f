"""Oracle: density matrices, Mulliken charges/spins and their first-order
response, by dense eigendecomposition in FP64.

Test infrastructure only (see oracle/__init__.py).

* Eq. D_min: D^sigma = [exp(beta (H^sigma - mu I)) + I]^{-1} (the beta = 1/kT
  missing from the printed exponent is restored), one chemical potential mu
  for both spins fixed by sum_sigma Tr D^sigma = N_e (the constraint written
  with Eqs. D_min, directBO, ShadowULatte).  Computed here by definition:
  H = C diag(eps) C^T, D = C diag(f(eps - mu)) C^T.
* Mulliken charges with S = I (Sec. III.A): per spin,
  q^sigma_I = sum_{i in I} (D^sigma - D0^sigma)_ii; q_I = q^up + q^dn and
  m_I = q^up - q^dn.  The extended-vector layout is [q^up; q^dn] (Sec. II.G).
* Eq. fv: the directional derivative q_v = d q[n + lambda v]/d lambda at 0.
  A direction v changes the per-atom shifts by
  dh_sigma = gamma (v_up + v_dn) + sigma (W/2)(v_up - v_dn); first-order
  perturbation theory in the eigenbasis gives
  dD' = F o (dH' - dmu I), F_ab = (f_a - f_b)/(eps_a - eps_b) (f' on the
  diagonal), with the common dmu fixed by sum_sigma Tr dD = 0.
* Eq. RegJacobian: J = df/dn with f = q - n, so column j of J is q_{e_j} - e_j.
"""
from __future__ import annotations

import numpy as np

from . import model

NORB = model.NORB


def fermi(x, beta):
    """f(x) = 1 / (1 + exp(beta x)), evaluated without overflow."""
    x = np.asarray(x, dtype=np.float64)
    z = beta * x
    out = np.empty_like(z)
    pos = z > 0
    ez = np.exp(-z[pos])
    out[pos] = ez / (1.0 + ez)
    out[~pos] = 1.0 / (1.0 + np.exp(z[~pos]))
    return out


def fermi_divided_differences(eps, mu, beta):
    """F_ab = (f(eps_a - mu) - f(eps_b - mu)) / (eps_a - eps_b), F_aa = f'(eps_a - mu).

    Uses the identity f(x) = (1 - tanh(beta x / 2)) / 2, which gives
    f_a - f_b = -sinh(h_a - h_b) / (2 cosh(h_a) cosh(h_b)) with h = beta x / 2,
    so F_ab = -(beta/4) sinhc(h_a - h_b) / (cosh(h_a) cosh(h_b)),
    sinhc(z) = sinh(z)/z.  It is evaluated in log space (ln sinhc and
    ln cosh), so nothing overflows and no nearly equal numbers are
    subtracted; the diagonal reduces to f'(x) = -beta f (1 - f)."""
    x = np.asarray(eps, dtype=np.float64) - mu
    h = 0.5 * beta * x
    dz = np.abs(h[:, None] - h[None, :])
    small = dz < 1e-4
    dzs = np.where(small, 1.0, dz)
    ln_sinhc = np.where(small, dz * dz / 6.0,
                        dzs + np.log1p(-np.exp(-2.0 * dzs)) - np.log(2.0 * dzs))
    ah = np.abs(h)
    ln_cosh = ah + np.log1p(np.exp(-2.0 * ah)) - np.log(2.0)
    return -(0.25 * beta) * np.exp(ln_sinhc - ln_cosh[:, None] - ln_cosh[None, :])


class SpinChannel:
    """Eigendecomposition of one H_sigma."""

    def __init__(self, H):
        self.eps, self.C = np.linalg.eigh(H)


def electron_count(chans, mu, beta):
    return sum(float(np.sum(fermi(c.eps - mu, beta))) for c in chans)


def find_mu(chans, n_elec, beta, tol=1e-13, mu_guess=None):
    """Common chemical potential: bracketed bisection with Newton steps on
    N(mu) = sum_sigma sum_a f(eps_a - mu) = N_e (N is increasing in mu)."""
    eps_all = np.concatenate([c.eps for c in chans])
    lo, hi = eps_all.min() - 50.0 / beta, eps_all.max() + 50.0 / beta
    mu = 0.5 * (lo + hi) if mu_guess is None else float(mu_guess)
    for _ in range(500):
        f = fermi(eps_all - mu, beta)
        N = float(np.sum(f))
        dN = float(np.sum(beta * f * (1.0 - f)))
        err = N - n_elec
        if abs(err) < tol * max(1.0, n_elec):
            return mu
        if err > 0:
            hi = mu
        else:
            lo = mu
        mu_new = mu - err / dN if dN > 0 else 0.5 * (lo + hi)
        if not (lo < mu_new < hi):
            mu_new = 0.5 * (lo + hi)
        mu = mu_new
    raise RuntimeError("chemical potential search did not converge")


class Density:
    """D_up, D_dn, mu, Mulliken q (2 N_at) for given H0, gamma and n."""

    def __init__(self, H0, gamma, n, p, mu_guess=None):
        self.p = p
        self.beta = 1.0 / p.kT
        self.gamma = gamma
        self.nat = gamma.shape[0]
        self.n = np.asarray(n, dtype=np.float64).copy()
        Hu, Hd = model.hamiltonians(H0, self.n, gamma, p)
        self.H = (Hu, Hd)
        self.chans = (SpinChannel(Hu), SpinChannel(Hd))
        self.n_elec = p.n_elec_per_atom * self.nat
        self.mu = find_mu(self.chans, self.n_elec, self.beta, mu_guess=mu_guess)
        self.occ = tuple(fermi(c.eps - self.mu, self.beta) for c in self.chans)
        # 1 - f evaluated directly as f(-x), exact for nearly full states
        self.occ_c = tuple(fermi(self.mu - c.eps, self.beta) for c in self.chans)
        self.D = tuple((c.C * f) @ c.C.T for c, f in zip(self.chans, self.occ))
        d0 = model.d0_diag(p)
        self.q_spin = tuple(
            (np.diag(D).reshape(self.nat, NORB) - d0).sum(axis=1) for D in self.D)

    @property
    def q(self):
        """Extended-vector layout [q_up; q_dn]."""
        return np.concatenate(self.q_spin)

    @property
    def charge(self):
        return self.q_spin[0] + self.q_spin[1]

    @property
    def spin(self):
        return self.q_spin[0] - self.q_spin[1]

    def residual(self):
        return self.q - self.n

    def response(self, v):
        """q_v = dq[n + lambda v]/dlambda (Eq. fv) by eigenbasis perturbation
        theory with a common dmu; returns (q_v [2 N_at], dmu)."""
        v = np.asarray(v, dtype=np.float64)
        nat = self.nat
        dh_up, dh_dn = model.spin_potentials(v, self.gamma, self.p)
        if not hasattr(self, "_F"):
            self._F = tuple(fermi_divided_differences(c.eps, self.mu, self.beta)
                            for c in self.chans)
        Fs, dHs = self._F, []
        for c, dh in zip(self.chans, (dh_up, dh_dn)):
            dhe = np.repeat(dh, NORB)
            dHs.append(c.C.T @ (dhe[:, None] * c.C))
        num = sum(float(np.sum(np.diag(F) * np.diag(dH))) for F, dH in zip(Fs, dHs))
        den = sum(float(np.sum(np.diag(F))) for F in Fs)
        dmu = num / den
        qv = []
        for c, F, dH in zip(self.chans, Fs, dHs):
            dDp = F * (dH - dmu * np.eye(dH.shape[0]))
            dD = c.C @ dDp @ c.C.T
            qv.append(np.diag(dD).reshape(nat, NORB).sum(axis=1))
        return np.concatenate(qv), dmu

    def fv(self, v):
        """f_v = q_v - v = J v (Eq. fv)."""
        return self.response(v)[0] - np.asarray(v)

    def jacobian(self):
        """Full 2N_at x 2N_at Jacobian J_ij = df_i/dn_j (Eq. RegJacobian),
        column by column from unit directions."""
        m = 2 * self.nat
        J = np.empty((m, m))
        for j in range(m):
            e = np.zeros(m)
            e[j] = 1.0
            J[:, j] = self.fv(e)
        return J

    def entropy_term(self):
        """kT sum_sigma sum_a [f ln f + (1-f) ln(1-f)] (Eq. Entropy times T_e,
        with the sign that makes f_FD the stationary point)."""
        tot = 0.0
        for f, g in zip(self.occ, self.occ_c):
            with np.errstate(divide="ignore", invalid="ignore"):
                a = np.where(f > 0, f * np.log(f), 0.0)
                b = np.where(g > 0, g * np.log(g), 0.0)
            tot += float(np.sum(a + b))
        return self.p.kT * tot


def density(R, cell, n, p, mu_guess=None):
    """Convenience: build H0 and gamma, then the density for n."""
    H0 = model.build_h0(R, cell, p)
    G = model.gamma_matrix(R, cell, p)
    return Density(H0, G, n, p, mu_guess=mu_guess)
