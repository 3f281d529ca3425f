"""The paper-general model on the GPU (fp64 form): non-orthogonal basis
(overlap S, Z = S^{-1/2} by Newton-Schulz on the device, H_perp = Z H Z,
D = Z D_perp Z) and l-resolved charges and spins with l-dependent Stoner
parameters (Sec. II.C, Sec. III.A), against the general oracle
(generalized eigenproblem, oracle/general.py).

* 16 atoms (144 orbitals) and 54 atoms (486 orbitals, ragged 64-tiles):
  mu, the shell-resolved occupations, a response direction, the forces
  (with the overlap derivative terms) and every energy term.
* The Krylov kernel K f (Eq. mIJacobian) at the 16-atom start.
* Ten sXL-BOMD steps of the 16-atom cell from its unconverged start
  (K0 = -I): positions, velocities and n step by step.
Tolerances: the fp64 form's 1e-10 e and 1e-8 eV/A.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dynamics, general, kernel, model  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def sxl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


@pytest.mark.parametrize("wname", ["fe16_general", "fe54_general"])
def test_general_density_response_forces(sxl, wname):
    w = getattr(wl, wname)()
    p, nat = w.params, w.n_atoms
    d = general.density(w.R, w.cell, w.n0, p)
    ctx = sxl.Context(p, nat, w.cell, "fp64")
    q, mu = ctx.density(w.R, w.n0)
    q = q.cpu().numpy()
    assert q.size == 6 * nat
    print(f"{wname}: |dq| {np.abs(q - d.q).max():.2e} |dmu| {abs(mu - d.mu):.2e}")
    assert abs(mu - d.mu) < 1e-9
    assert np.abs(q - d.q).max() < 1e-10
    D = ctx.density_matrix().cpu().numpy()
    assert np.abs(D - np.stack(d.D)).max() < 1e-10
    v = wl.random_direction(3 * nat, 5)
    qv, dmu = ctx.response(v)
    qv_o, dmu_o = d.response(v)
    print(f"{wname}: |dq_v| {np.abs(qv.cpu().numpy() - qv_o).max():.2e}")
    assert np.abs(qv.cpu().numpy() - qv_o).max() < 1e-9
    assert abs(dmu - dmu_o) < 1e-9
    F, en = ctx.forces(w.R, w.n0, energies=True)
    F_o = general.forces(d, w.R, w.cell)
    e_o = general.shadow_energy(d, model.build_h0(w.R, w.cell, p),
                                model.repulsive_energy(w.R, w.cell, p))
    print(f"{wname}: |dF| {np.abs(F.cpu().numpy() - F_o).max():.2e} "
          f"dU {abs(en['U'] - e_o['U']):.2e}")
    assert np.abs(F.cpu().numpy() - F_o).max() < 1e-8
    for k in ("band", "coul", "spin", "entropy", "rep"):
        assert abs(en[k] - e_o[k]) < 1e-8 * nat, (k, en[k], e_o[k])
    assert abs(en["U"] - e_o["U"]) < 1e-8 * nat
    ctx.close()


def test_general_krylov_kernel(sxl):
    w = wl.fe16_general()
    p, nat = w.params, w.n_atoms
    d = general.density(w.R, w.cell, w.n0, p)
    K0 = -np.eye(6 * nat)
    Kf_o, info = kernel.krylov_kernel(d, K0, p.krylov_rank)
    ctx = sxl.Context(p, nat, w.cell, "fp64")
    Kf, q, rel = ctx.krylov(w.R, w.n0, p.krylov_rank)
    assert np.abs(Kf.cpu().numpy() - Kf_o).max() < 1e-9 * max(1.0, np.abs(Kf_o).max())
    assert abs(rel - info["rel"]) < 1e-9
    ctx.close()


def test_general_xlbomd_steps(sxl):
    w = wl.fe16_general()
    p, nat = w.params, w.n_atoms
    md = dynamics.XLBOMD(w.R, w.V, w.cell, w.n0, p, -np.eye(6 * nat), general_model=True)
    ctx = sxl.Context(p, nat, w.cell, "fp64")
    ctx.set_state(w.R, w.V, np.tile(w.n0, (p.kmax + 1, 1)), md.mu)
    for _ in range(10):
        st_o = md.step()
        st = ctx.step(1)[0]
        R, V, nh, mu = ctx.get_state()
        np.testing.assert_allclose(R.cpu().numpy(), md.R, atol=1e-10)
        np.testing.assert_allclose(V.cpu().numpy(), md.V, atol=1e-11)
        np.testing.assert_allclose(nh.cpu().numpy()[0], md.nhist[0], atol=1e-9)
        assert abs(mu - st_o["mu"]) < 1e-9
        assert abs(st[0] - st_o["Etot"]) < 1e-8 * nat
    ctx.close()
