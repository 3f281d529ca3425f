"""Oracle: integration of the sXL-BOMD equations of motion and the SCF with
the kernel quasi-Newton mixer.

Test infrastructure only (see oracle/__init__.py).

Eq. Integration (modified leapfrog velocity Verlet with dissipation):
  V(t + dt/2) = V(t) + dt/2 a(t)
  R(t + dt)   = R(t) + dt V(t + dt/2)
  n(t + dt)   = 2 n(t) - n(t - dt) + dt^2 n''(t) + alpha sum_{k=0}^{kmax} c_k n(t - k dt)
  V(t + dt)   = V(t + dt/2) + dt/2 a(t + dt)
with dt^2 n''(t) = -kappa K f(t) (Eq. Eq_Mot2, kappa = dt^2 w^2) and K f from the
low-rank Krylov kernel (Eq. mIJacobian).  The kappa, alpha, c_k of the cited
integrator paper are not in the text; the values used are parameters
(kmax = 5: kappa 1.82, alpha 0.018, c = -6, 14, -8, -3, 4, -1).
Initialization (Sec. II.E): every n(t0 - k dt) is the converged SCF n at t0.

Eq. QN: n_new = n_old - K (q[n_old] - n_old) with the Krylov kernel; linear
mixing (coefficient 0.06) until the residual RMS drops below 0.05, then the
exact kernel J^{-1} at that point is taken as K0 and kept (Sec. III.C,
Fig. SCF caption).  Ranks are adaptive (stop once the relative least-squares
residual is below 0.1, at most `rank`).

The comparison mixers of Fig. SCF: plain linear mixing (0.06) throughout,
and Pulay's DIIS switched on at the same 0.05 threshold.  DIIS keeps the last
`diis_hist` pairs (n_i, f_i), takes the coefficients c minimizing
|sum c_i f_i| subject to sum c_i = 1 (Lagrange system with B_ij = f_i . f_j)
and sets n_new = sum c_i (n_i + diis_mix f_i); the paper gives neither the
history length nor the mixing, so 8 and 0.1 are parameters.
"""
from __future__ import annotations

import numpy as np

from . import electronic, energy, general, kernel, model

KB = 8.617333262e-5          # eV / K
MVV_TO_EV = 103.642696562    # amu A^2 / fs^2 in eV


def kinetic_energy(V, mass):
    return 0.5 * mass * MVV_TO_EV * float(np.sum(V * V))


def temperature(V, mass):
    nat = V.shape[0]
    return 2.0 * kinetic_energy(V, mass) / ((3 * nat - 3) * KB)


def rms(x):
    return float(np.sqrt(np.mean(np.asarray(x) ** 2)))


def diis_update(ns, fs, mix):
    """Pulay step from the histories ns, fs (lists of vectors)."""
    m = len(fs)
    B = np.empty((m + 1, m + 1))
    for i in range(m):
        for j in range(m):
            B[i, j] = fs[i] @ fs[j]
    B[m, :m] = B[:m, m] = 1.0
    B[m, m] = 0.0
    rhs = np.zeros(m + 1)
    rhs[m] = 1.0
    c = np.linalg.solve(B, rhs)[:m]
    return sum(ci * (ni + mix * fi) for ci, ni, fi in zip(c, ns, fs))


def scf(R, cell, n0, p, tol=1e-8, max_iter=200, rank=None, lin_mix=0.06,
        kernel_on=0.05, rel_tol=0.1, return_history=False, mixer="kernel",
        diis_hist=8, diis_mix=0.1):
    """SCF with linear mixing, then the Krylov quasi-Newton kernel mixer
    (mixer="kernel"), Pulay DIIS ("diis") or linear mixing only ("linear")."""
    rank = p.krylov_rank if rank is None else rank
    H0 = model.build_h0(R, cell, p)
    G = model.gamma_matrix(R, cell, p)
    n = np.array(n0, dtype=np.float64)
    K0 = None
    mu = None
    hist = []
    dn, df = [], []
    diis_on = False
    for it in range(max_iter):
        dens = electronic.Density(H0, G, n, p, mu_guess=mu)
        mu = dens.mu
        f = dens.residual()
        r = rms(f)
        hist.append(r)
        if r < tol:
            out = dict(n=n, iters=it, rms=r, K0=K0, mu=mu, dens=dens)
            if return_history:
                out["history"] = hist
            return out
        if mixer == "linear" or (mixer == "diis" and not diis_on and r >= kernel_on) or \
                (mixer == "kernel" and K0 is None and r >= kernel_on):
            n = n + lin_mix * f
            continue
        if mixer == "diis":
            diis_on = True
            dn.append(n.copy())
            df.append(f.copy())
            dn, df = dn[-diis_hist:], df[-diis_hist:]
            n = diis_update(dn, df, diis_mix)
            continue
        if K0 is None:
            K0 = kernel.exact_kernel(dens)
        Kf, _ = kernel.krylov_kernel(dens, K0, rank, f=f, rel_tol=rel_tol)
        n = n - Kf
    raise RuntimeError(f"SCF did not converge, rms={hist[-1]:.3e}")


class XLBOMD:
    """State and time stepping of Eq. Integration."""

    def __init__(self, R, V, cell, n_star, p, K0, mu=None, general_model=False, recycle=False):
        """general_model: the non-orthogonal, l-resolved model of
        oracle/general.py in place of the orthogonal per-atom one.
        recycle: after the first evaluation, the kernel of each step is the
        recycled-subspace variant over the previous step's directions
        (kernel.krylov_kernel_subspace, a build choice, not the paper's)."""
        self.p = p
        self.general_model = general_model
        self.recycle = recycle
        self.Vrec = None
        self.cell = np.asarray(cell, dtype=np.float64)
        self.R = np.array(R, dtype=np.float64)
        self.V = np.array(V, dtype=np.float64)
        self.K0 = K0
        self.nhist = [np.array(n_star, dtype=np.float64) for _ in range(p.kmax + 1)]
        self.mu = mu
        self._evaluate()

    def _evaluate(self):
        p = self.p
        H0 = model.build_h0(self.R, self.cell, p)
        G = model.gamma_matrix(self.R, self.cell, p)
        n = self.nhist[0]
        if self.general_model:
            S = general.overlap(self.R, self.cell, p)
            self.dens = general.GDensity(H0, S, G, n, p, mu_guess=self.mu)
            self.F = general.forces(self.dens, self.R, self.cell)
            self.E = general.shadow_energy(self.dens, H0,
                                           model.repulsive_energy(self.R, self.cell, p))
        else:
            self.dens = electronic.Density(H0, G, n, p, mu_guess=self.mu)
            self.F = energy.forces(self.dens, self.R, self.cell)
            self.E = energy.shadow_energy(self.dens, H0,
                                          model.repulsive_energy(self.R, self.cell, p))
        self.mu = self.dens.mu
        if self.recycle and self.Vrec is not None:
            self.Kf, self.kinfo = kernel.krylov_kernel_subspace(
                self.dens, self.K0, [self.Vrec[:, j] for j in range(self.Vrec.shape[1])],
                p.krylov_rank)
        else:
            self.Kf, self.kinfo = kernel.krylov_kernel(self.dens, self.K0, p.krylov_rank)
        if self.recycle:
            self.Vrec = self.kinfo["V"]

    def accel(self):
        return self.F / (self.p.mass_amu * MVV_TO_EV)

    def step(self):
        p = self.p
        dt = p.dt_fs
        self.V = self.V + 0.5 * dt * self.accel()
        self.R = self.R + dt * self.V
        n_new = 2.0 * self.nhist[0] - self.nhist[1] - p.kappa * self.Kf
        n_new = n_new + p.alpha * sum(ck * self.nhist[k] for k, ck in enumerate(p.c))
        self.nhist = [n_new] + self.nhist[:-1]
        self._evaluate()
        self.V = self.V + 0.5 * dt * self.accel()
        return self.stats()

    def stats(self):
        ke = kinetic_energy(self.V, self.p.mass_amu)
        return dict(Etot=self.E["U"] + ke, U=self.E["U"], KE=ke,
                    T=temperature(self.V, self.p.mass_amu),
                    rms=rms(self.dens.residual()), mu=self.mu)


class BOMD:
    """Regular Born-Oppenheimer MD, the comparison of Sec. IV: velocity
    Verlet with the forces of the SCF ground state, the SCF at each step
    started from the previous step's converged n and mixed with `mixer`
    (scf above) to RMS(q - n) < tol."""

    def __init__(self, R, V, cell, n0, p, tol=1e-8, mixer="diis", max_iter=400, mu=None):
        self.p = p
        self.cell = np.asarray(cell, dtype=np.float64)
        self.R = np.array(R, dtype=np.float64)
        self.V = np.array(V, dtype=np.float64)
        self.tol, self.mixer, self.max_iter = tol, mixer, max_iter
        self.n = np.array(n0, dtype=np.float64)
        self.mu = mu
        self.scf_iters = []
        self._evaluate()

    def _evaluate(self):
        res = scf(self.R, self.cell, self.n, self.p, tol=self.tol, max_iter=self.max_iter,
                  mixer=self.mixer)
        self.n, self.mu, self.dens = res["n"], res["mu"], res["dens"]
        self.scf_iters.append(res["iters"])
        self.F = energy.forces(self.dens, self.R, self.cell)
        H0 = model.build_h0(self.R, self.cell, self.p)
        self.E = energy.shadow_energy(self.dens, H0,
                                      model.repulsive_energy(self.R, self.cell, self.p))

    def step(self):
        dt = self.p.dt_fs
        acc = self.F / (self.p.mass_amu * MVV_TO_EV)
        self.V = self.V + 0.5 * dt * acc
        self.R = self.R + dt * self.V
        self._evaluate()
        self.V = self.V + 0.5 * dt * self.F / (self.p.mass_amu * MVV_TO_EV)
        ke = kinetic_energy(self.V, self.p.mass_amu)
        return dict(Etot=self.E["U"] + ke, T=temperature(self.V, self.p.mass_amu),
                    rms=rms(self.dens.residual()), mu=self.mu, scf_iters=self.scf_iters[-1])
