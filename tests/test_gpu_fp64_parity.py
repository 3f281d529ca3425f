"""FP64 CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Tolerances (FP64 form): charges and spins 1e-10 e, forces 1e-8 eV/A; the
intermediate objects (H, D, q_v, Kf) are held to comparable absolute bounds.
Sizes: 16 atoms (N = 144, a ragged 2.25 GEMM tiles) and 54 atoms (N = 486,
7.6 tiles)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dynamics, electronic, energy, kernel, model  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl
    return sxl


def _ctx(sxl, w, **kw):
    return sxl.Context(w.params, w.n_atoms, w.cell, "fp64", **kw)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def case16(lib):
    w = wl.fe16()
    d = electronic.density(w.R, w.cell, w.n0, w.params)
    return w, d


def test_hamiltonian_matches(lib, case16):
    w, d = case16
    ctx = _ctx(lib, w)
    H = _np(ctx.hamiltonian(w.R, w.n0))
    np.testing.assert_allclose(H[0], d.H[0], atol=1e-12)
    np.testing.assert_allclose(H[1], d.H[1], atol=1e-12)


@pytest.mark.parametrize("which", ["fe16", "cell54"])
def test_density_charges_mu(lib, which):
    w = wl.fe16() if which == "fe16" else wl.make_cell(3, seed=54, name="cell54")
    d = electronic.density(w.R, w.cell, w.n0, w.params)
    ctx = _ctx(lib, w)
    q, mu = ctx.density(w.R, w.n0)
    assert abs(mu - d.mu) < 1e-10
    np.testing.assert_allclose(_np(q), d.q, atol=1e-10)
    D = _np(ctx.density_matrix())
    np.testing.assert_allclose(D[0], d.D[0], atol=1e-10)
    np.testing.assert_allclose(D[1], d.D[1], atol=1e-10)


def test_response_matches(lib, case16):
    w, d = case16
    ctx = _ctx(lib, w)
    ctx.density(w.R, w.n0)
    for seed in (3, 4):
        v = wl.random_direction(16, seed)
        qv, dmu = ctx.response(v)
        qv_o, dmu_o = d.response(v)
        np.testing.assert_allclose(_np(qv), qv_o, atol=1e-9)
        assert abs(dmu - dmu_o) < 1e-9


def test_krylov_kernel_matches(lib, case16):
    w, d = case16
    ctx = _ctx(lib, w)
    Kf, q, rel = ctx.krylov(w.R, w.n0, 4)
    Kf_o, info = kernel.krylov_kernel(d, -np.eye(32), 4)
    np.testing.assert_allclose(_np(q), d.q, atol=1e-10)
    np.testing.assert_allclose(_np(Kf), Kf_o, atol=1e-8 * max(1.0, np.abs(Kf_o).max()))
    assert abs(rel - info["rel"]) < 1e-7


def test_exact_k0_jacobian(lib, case16):
    w, d = case16
    ctx = _ctx(lib, w)
    ctx.density(w.R, w.n0)
    J = _np(ctx.build_exact_k0(want_J=True))
    np.testing.assert_allclose(J, d.jacobian(), atol=1e-9)
    # with the exact preconditioner installed, rank 1 gives J^{-1} f
    Kf, _, _ = ctx.krylov(w.R, w.n0, 1)
    np.testing.assert_allclose(_np(Kf), np.linalg.solve(d.jacobian(), d.residual()), atol=1e-8)


def test_forces_and_energy_terms(lib, case16):
    w, d = case16
    ctx = _ctx(lib, w)
    F, en = ctx.forces(w.R, w.n0)
    F_o = energy.forces(d, w.R, w.cell)
    np.testing.assert_allclose(_np(F), F_o, atol=1e-8)
    H0 = model.build_h0(w.R, w.cell, w.params)
    e_o = energy.shadow_energy(d, H0, model.repulsive_energy(w.R, w.cell, w.params))
    for k in ("band", "coul", "spin", "rep"):
        assert abs(en[k] - e_o[k]) < 1e-8, k
    # electronic entropy through the chain log-determinants: 1e-8 eV/atom
    assert abs(en["entropy"] - e_o["entropy"]) < 1e-8 * w.n_atoms, (en["entropy"], e_o["entropy"])
    assert abs(en["U"] - e_o["U"]) < 1e-8 * w.n_atoms


def test_scf_fixed_point(lib):
    w = wl.fe16()
    ctx = _ctx(lib, w)
    n, iters, rms = ctx.scf(w.R, w.n0, tol=1e-9)
    res = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-9)
    assert rms < 1e-9
    np.testing.assert_allclose(_np(n), res["n"], atol=1e-8)


def test_xlbomd_trajectory_matches_oracle(lib):
    """The 16-atom cell's full run, 100 sXL-BOMD steps from the SCF point
    (exact K0, rank 4): positions, velocities, n, temperature, RMS(q - n)
    and mu follow the oracle step by step."""
    w = wl.fe16()
    res = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-10)
    md = dynamics.XLBOMD(w.R, w.V, w.cell, res["n"], w.params, res["K0"], mu=res["mu"])
    ctx = _ctx(lib, w)
    ctx.set_k0(res["K0"])
    nh = np.tile(res["n"], (w.params.kmax + 1, 1))
    ctx.set_state(w.R, w.V, nh, res["mu"])
    for step in range(100):
        st_o = md.step()
        st = ctx.step(1)[0]
        R, V, nhg, mu = ctx.get_state()
        np.testing.assert_allclose(_np(R), md.R, atol=1e-10)
        np.testing.assert_allclose(_np(V), md.V, atol=1e-11)
        np.testing.assert_allclose(_np(nhg)[0], md.nhist[0], atol=1e-9)
        assert abs(mu - st_o["mu"]) < 1e-9
        assert abs(st[1] - st_o["T"]) < 1e-6
        assert abs(st[2] - st_o["rms"]) < 1e-9


@pytest.mark.parametrize("sym", [False, True])
def test_gemm_f64_against_numpy(lib, sym):
    """The fp64 form's product (k_gemm_f64, 64 x 64 tiles) on the 16-atom
    size N = 144 (two full tiles and a ragged one), with the epilogue
    alpha A B^T + beta E + gamma I; symmetric mode mirrors the upper tiles."""
    w = wl.fe16()
    ctx = _ctx(lib, w)
    n = w.n_orb
    rng = np.random.default_rng(8)
    A = rng.normal(size=(2, n, n))
    B = A.copy() if sym else rng.normal(size=(2, n, n))
    E = rng.normal(size=(2, n, n))
    E = E + np.transpose(E, (0, 2, 1))
    C = ctx.gemm_f64(A, B, E, alpha=0.7, beta=-1.5, gamma=2.0, sym=sym).cpu().numpy()
    ref = 0.7 * np.einsum("bij,bkj->bik", A, B) - 1.5 * E + 2.0 * np.eye(n)
    assert np.abs(C - ref).max() < 1e-12 * np.abs(ref).max()
    if sym:
        assert np.array_equal(C, np.transpose(C, (0, 2, 1)))
    ctx.close()
