"""Pins of the oracle's Krylov kernel (Eq. mIJacobian), SCF (Eq. QN), shadow
energy and forces (Eqs. ShadowELatte, EqMot) and integrator (Eq. Integration)."""
import numpy as np
import pytest

from oracle import dynamics, electronic, energy, kernel, model
from paper_2303_03529_gb300 import workload as wl


@pytest.fixture(scope="module")
def dens16():
    w = wl.fe16()
    return w, electronic.density(w.R, w.cell, w.n0, w.params)


def test_full_rank_krylov_is_exact_inverse_jacobian(dens16):
    """With a complete basis Eq. mIJacobian is an identity: K f = J^{-1} f."""
    w, d = dens16
    J = d.jacobian()
    f = d.residual()
    for K0 in (-np.eye(32), np.diag(-1.0 / (1.0 + np.arange(32) / 10.0))):
        Kf, info = kernel.krylov_kernel(d, K0, rank=32)
        np.testing.assert_allclose(Kf, np.linalg.solve(J, f), atol=1e-9)
    # exact preconditioner: rank 1 already exact
    Kf1, info = kernel.krylov_kernel(d, np.linalg.inv(J), rank=1)
    np.testing.assert_allclose(Kf1, np.linalg.solve(J, f), atol=1e-10)


def test_no_coupling_gives_minus_identity():
    """gamma = 0 and W = 0 (U -> 0 via coulomb_k = 0): q does not depend on n,
    so J = -I and the rank-1 Krylov kernel with K0 = -I is exact."""
    p = wl.ModelParams(coulomb_k=0.0, U=1e-300, W=0.0)
    w = wl.make_cell(2, seed=2, params=p)
    H0 = model.build_h0(w.R, w.cell, p)
    G = np.zeros((16, 16))
    d = electronic.Density(H0, G, w.n0, p)
    np.testing.assert_allclose(d.jacobian(), -np.eye(32), atol=1e-13)
    Kf, _ = kernel.krylov_kernel(d, -np.eye(32), rank=1)
    np.testing.assert_allclose(Kf, -d.residual(), atol=1e-13)


def test_krylov_basis_is_orthonormal_and_lsq_optimal(dens16):
    w, d = dens16
    K0 = -np.eye(32)
    Kf, info = kernel.krylov_kernel(d, K0, rank=4)
    V = info["V"]
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)
    FT = info["FT"]
    ft = K0 @ d.residual()
    r = FT @ info["c"] - ft
    np.testing.assert_allclose(FT.T @ r, 0.0, atol=1e-12)   # normal equations


def test_scf_fixed_point():
    w = wl.fe16()
    res = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-9)
    d = electronic.density(w.R, w.cell, res["n"], w.params)
    assert dynamics.rms(d.residual()) < 1e-9
    assert res["K0"] is not None   # the kernel mixer took over


def test_diis_single_entry_is_linear_mixing():
    rng = np.random.default_rng(3)
    n, f = rng.standard_normal(7), rng.standard_normal(7)
    np.testing.assert_allclose(dynamics.diis_update([n], [f], 0.3), n + 0.3 * f, atol=1e-15)


def test_diis_two_entries_closed_form():
    """m = 2: c1 minimizes |c1 f1 + (1 - c1) f2|, c1 = f2.(f2 - f1) / |f1 - f2|^2."""
    rng = np.random.default_rng(4)
    n1, n2, f1, f2 = (rng.standard_normal(6) for _ in range(4))
    c1 = f2 @ (f2 - f1) / ((f1 - f2) @ (f1 - f2))
    want = c1 * (n1 + 0.1 * f1) + (1 - c1) * (n2 + 0.1 * f2)
    np.testing.assert_allclose(dynamics.diis_update([n1, n2], [f1, f2], 0.1), want, atol=1e-13)


def test_diis_solves_affine_residual_exactly():
    """For f(n) = b - A n and dim + 1 affinely independent points, sum c_i f_i
    = 0 is reachable, so the Pulay step lands on A^{-1} b for any mixing."""
    rng = np.random.default_rng(5)
    d = 5
    M = rng.standard_normal((d, d))
    A = M @ M.T + d * np.eye(d)
    b = rng.standard_normal(d)
    ns = [rng.standard_normal(d) for _ in range(d + 1)]
    fs = [b - A @ x for x in ns]
    for mix in (0.0, 0.1, 0.7):
        np.testing.assert_allclose(dynamics.diis_update(ns, fs, mix), np.linalg.solve(A, b),
                                   atol=1e-10)


def test_scf_mixers_reach_the_same_fixed_point():
    """DIIS and kernel mixing converge to one q[n] = n; the kernel mixer needs
    the fewest iterations, linear mixing (0.06) is still far from converged
    after as many iterations as DIIS took (the ordering of Fig. SCF)."""
    w = wl.fe16()
    res = {m: dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-8, max_iter=400, mixer=m)
           for m in ("kernel", "diis")}
    np.testing.assert_allclose(res["diis"]["n"], res["kernel"]["n"], atol=1e-7)
    assert res["kernel"]["iters"] < res["diis"]["iters"]
    with pytest.raises(RuntimeError):
        dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-8, max_iter=res["diis"]["iters"],
                     mixer="linear")


def _energy_at(w, R, n):
    d = electronic.density(R, w.cell, n, w.params)
    e_rep = model.repulsive_energy(R, w.cell, w.params)
    return energy.shadow_energy(d, model.build_h0(R, w.cell, w.params), e_rep)["U"], d


def test_forces_are_minus_gradient_at_constant_n(dens16):
    w, d = dens16
    F = energy.forces(d, w.R, w.cell)
    assert np.abs(F.sum(axis=0)).max() < 1e-10
    h = 1e-4
    for atom, comp in ((0, 0), (5, 1), (11, 2)):
        Rp = w.R.copy()
        Rp[atom, comp] += h
        Rm = w.R.copy()
        Rm[atom, comp] -= h
        fd = -(_energy_at(w, Rp, w.n0)[0] - _energy_at(w, Rm, w.n0)[0]) / (2 * h)
        assert abs(F[atom, comp] - fd) < 1e-6


def test_entropy_sign_makes_fd_stationary(dens16):
    """The shadow energy, as a function of occupations at fixed eigenvectors,
    is stationary at f_FD under charge-conserving variations."""
    w, d = dens16
    p = w.params
    H0 = model.build_h0(w.R, w.cell, p)
    rng = np.random.default_rng(0)
    wts = [f * (1 - f) for f in d.occ]
    g = [rng.normal(size=144) * wt for wt in wts]
    # remove the component that changes the electron count
    a = sum(x.sum() for x in g) / sum(wt.sum() for wt in wts)
    g = [x - a * wt for x, wt in zip(g, wts)]

    def U_of(lam):
        dd = electronic.Density.__new__(electronic.Density)
        dd.__dict__.update(d.__dict__)
        occ = tuple(f + lam * gg for f, gg in zip(d.occ, g))
        dd.occ = occ
        dd.occ_c = tuple(1.0 - o for o in occ)
        dd.D = tuple((c.C * o) @ c.C.T for c, o in zip(d.chans, occ))
        d0 = model.d0_diag(p)
        dd.q_spin = tuple((np.diag(D).reshape(16, 9) - d0).sum(axis=1) for D in dd.D)
        return energy.shadow_energy(dd, H0)["U"]

    lam = 1e-4
    slope = (U_of(lam) - U_of(-lam)) / (2 * lam)
    assert abs(sum(x.sum() for x in g)) < 1e-12
    assert abs(slope) < 1e-7
    # the opposite entropy sign would not be stationary
    scale = sum(float(np.sum(gg * (np.log(f) - np.log(fc))))
                for gg, f, fc in zip(g, d.occ, d.occ_c))
    assert abs(2 * p.kT * scale) > 1e-3


def test_integrator_coefficients_and_stability():
    p = wl.ModelParams()
    c = np.array(p.c)
    assert abs(c.sum()) < 1e-15
    assert abs(np.dot(np.arange(len(c)), c)) < 1e-15
    # error recurrence e+ = (2 - kappa) e - e- + alpha sum c_k e_k
    K = p.kmax
    poly = np.zeros(K + 2)
    poly[0] = 1.0
    poly[1] = -(2.0 - p.kappa)
    poly[2] = 1.0
    for k, ck in enumerate(c):
        poly[1 + k] -= p.alpha * ck
    roots = np.roots(poly)
    assert np.max(np.abs(roots)) <= 1.0 + 1e-9


def test_integrator_keeps_linear_sequence():
    """Without kernel force, a linear-in-time n is propagated exactly."""
    p = wl.ModelParams()
    hist = [np.array([1.0 - 0.1 * k, 2.0 + 0.3 * k]) for k in range(p.kmax + 1)]
    n_new = 2 * hist[0] - hist[1] + p.alpha * sum(ck * hist[k] for k, ck in enumerate(p.c))
    np.testing.assert_allclose(n_new, [1.1, 1.7], atol=1e-14)


@pytest.mark.slow
def test_shadow_energy_conservation_and_dt2_scaling():
    """16 atoms from the SCF point: the residual RMS and the energy
    fluctuation shrink about 4x when dt is halved (Sec. III.B)."""
    w = wl.fe16()
    res = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-10)
    out = {}
    for dt, nsteps in ((0.5, 40), (0.25, 80)):
        p = w.params.replace(dt_fs=dt)
        md = dynamics.XLBOMD(w.R, w.V, w.cell, res["n"], p, res["K0"], mu=res["mu"])
        e0 = md.stats()["Etot"]
        st = [md.step() for _ in range(nsteps)]
        E = np.array([s["Etot"] for s in st])
        out[dt] = (np.max(np.abs(E - e0)), np.sqrt(np.mean([s["rms"] ** 2 for s in st])))
    ratio_rms = out[0.5][1] / out[0.25][1]
    ratio_e = out[0.5][0] / out[0.25][0]
    assert 2.5 < ratio_rms < 6.0
    assert 2.0 < ratio_e < 8.0
    assert out[0.5][0] / 16 < 1e-3   # eV/atom fluctuation bound over 20 fs


def test_bomd_forces_are_minus_gradient_of_bo_energy():
    """At the SCF fixed point U(R, n) is stationary in n, so the constant-n
    forces of the converged state are -dE_BO/dR with E_BO(R) = U(R, n*(R))
    (the property regular BOMD relies on).  Richardson-extrapolated central
    differences of E_BO, each point converged with DIIS to 1e-11."""
    w = wl.fe16()
    p = w.params

    def e_bo(R):
        res = dynamics.scf(R, w.cell, w.n0, p, tol=1e-11, max_iter=600, mixer="diis")
        H0 = model.build_h0(R, w.cell, p)
        return energy.shadow_energy(res["dens"], H0, model.repulsive_energy(R, w.cell, p))["U"], res

    _, res0 = e_bo(w.R)
    F = energy.forces(res0["dens"], w.R, w.cell)
    for (a, c) in ((0, 0), (5, 1), (11, 2)):
        def d(h):
            Rp, Rm = w.R.copy(), w.R.copy()
            Rp[a, c] += h
            Rm[a, c] -= h
            return (e_bo(Rp)[0] - e_bo(Rm)[0]) / (2 * h)
        g = (4 * d(1e-3) - d(2e-3)) / 3
        assert abs(g + F[a, c]) < 1e-7, (a, c, g, F[a, c])


def test_subspace_kernel_full_basis_is_exact_inverse_jacobian(dens16):
    """The recycled-subspace variant over a complete candidate basis spans
    R^{2 N_at}: K f = J^{-1} f (J from unit-direction responses), whatever
    the candidates' order (f~ comes first, then 31 of the unit vectors fill
    the space)."""
    w, d = dens16
    J = d.jacobian()
    f = d.residual()
    rng = np.random.default_rng(1)
    cands = [np.eye(32)[i] for i in rng.permutation(32)]
    for K0 in (-np.eye(32), np.diag(-1.0 / (1.0 + np.arange(32) / 10.0))):
        Kf, info = kernel.krylov_kernel_subspace(d, K0, cands, rank=32)
        assert info["rank"] == 32
        np.testing.assert_allclose(Kf, np.linalg.solve(J, f), atol=1e-9)
        np.testing.assert_allclose(info["V"].T @ info["V"], np.eye(32), atol=1e-12)


def test_subspace_kernel_on_the_krylov_span_equals_the_krylov_kernel(dens16):
    """Candidates that span the paper's rank-m Krylov space give its kernel
    (the least-squares projection depends on the span only), and candidates
    already in the span of f~ are dropped."""
    w, d = dens16
    K0 = -np.eye(32)
    Kf_k, info_k = kernel.krylov_kernel(d, K0, rank=5)
    V = info_k["V"]
    mix = V @ np.array([[1.0, 0.2, 0.0, 0.3, 0.1], [0.0, 1.0, 0.4, 0.0, 0.2],
                        [0.5, 0.0, 1.0, 0.1, 0.0], [0.0, 0.3, 0.0, 1.0, 0.6],
                        [0.1, 0.0, 0.2, 0.0, 1.0]])
    cands = [mix[:, i] for i in range(5)]
    Kf_s, info_s = kernel.krylov_kernel_subspace(d, K0, cands, rank=5)
    assert info_s["rank"] == 5
    np.testing.assert_allclose(Kf_s, Kf_k, atol=1e-11)
    ft = K0 @ d.residual()
    Kf_1, info_1 = kernel.krylov_kernel_subspace(d, K0, [2.0 * ft, -ft], rank=5)
    assert info_1["rank"] == 1


def test_recycled_kernel_dynamics_match_the_krylov_kernel():
    """40 sXL-BOMD steps of the 16-atom cell from its SCF point with the
    recycled-subspace kernel stay on the same shadow surface as with the
    Krylov construction: the same energy spread and residual within a small
    factor, and trajectories that agree to far below the thermal scale
    (both kernels approximate the same J^-1)."""
    w = wl.fe16()
    p = w.params
    s = dynamics.scf(w.R, w.cell, w.n0, p, tol=1e-10)
    runs = {}
    for rec in (False, True):
        md = dynamics.XLBOMD(w.R, w.V, w.cell, s["n"], p, s["K0"], mu=s["mu"], recycle=rec)
        st = [md.step() for _ in range(40)]
        runs[rec] = (np.array([x["Etot"] for x in st]), np.array([x["rms"] for x in st]), md.R)
    (Ek, rk, Rk), (Er, rr, Rr) = runs[False], runs[True]
    spread = lambda E: (E.max() - E.min()) / w.n_atoms
    assert spread(Er) < 2.0 * spread(Ek) + 1e-7
    assert rr.max() < 2.0 * rk.max() + 1e-6
    assert np.abs(Rr - Rk).max() < 1e-4
