"""128-atom cell (4x4x4 bcc, 1152 orbitals x 2 spins, Krylov rank 6).

* SCF from the ferromagnetic start (m_I = 2 +- 0.1) with linear mixing 0.06,
  the exact K0 = J^{-1} built at the kernel switch and the Krylov
  quasi-Newton steps of Eq. QN, converged to RMS(q - n) < 1e-8; the oracle
  confirms q[n*] = n* at the GPU's n*.
* Three sXL-BOMD steps in the FP64 form against the oracle step by step,
  from the unconverged start with K0 = -I (a stress test of every stage:
  large residual, strong kernel action).
* Thirty mixed-precision (fp16) steps from the SCF point: bounded shadow
  energy and a residual that stays small (stability of the mixed form).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dynamics, electronic  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def sxl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


@pytest.fixture(scope="module")
def scf128(sxl):
    w = wl.fe128()
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, "fp64")
    n, iters, rms = ctx.scf(w.R, w.n0, tol=1e-8, max_iter=300)
    return w, n.cpu().numpy(), iters, rms


def test_scf_128_fixed_point(scf128):
    w, n, iters, rms = scf128
    assert rms < 1e-8
    d = electronic.density(w.R, w.cell, n, w.params)
    assert dynamics.rms(d.residual()) < 2e-8
    assert abs(np.sum(n)) < 1e-8   # neutral


def test_md_128_fp64_three_steps(sxl):
    w = wl.fe128()
    p = w.params
    md = dynamics.XLBOMD(w.R, w.V, w.cell, w.n0, p, -np.eye(256))
    ctx = sxl.Context(p, w.n_atoms, w.cell, "fp64")
    nh = np.tile(w.n0, (p.kmax + 1, 1))
    ctx.set_state(w.R, w.V, nh, md.mu)
    for _ in range(3):
        st_o = md.step()
        st = ctx.step(1)[0]
        R, V, nhg, mu = ctx.get_state()
        np.testing.assert_allclose(R.cpu().numpy(), md.R, atol=1e-10)
        np.testing.assert_allclose(V.cpu().numpy(), md.V, atol=1e-11)
        np.testing.assert_allclose(nhg.cpu().numpy()[0], md.nhist[0], atol=1e-9)
        assert abs(mu - st_o["mu"]) < 1e-9
        assert abs(st[0] - st_o["Etot"]) < 1e-8 * w.n_atoms


def test_md_128_mixed_stable(sxl, scf128):
    w, n_star, _, _ = scf128
    p = w.params
    ctx = sxl.Context(p, w.n_atoms, w.cell, "fp16", scf_keep_k0=1)
    _, mu = ctx.density(w.R, n_star)
    ctx.set_state(w.R, w.V, np.tile(n_star, (p.kmax + 1, 1)), mu)
    st = ctx.step(30)
    E = st[:, 0]
    print("mixed 128: dE/atom max", np.abs(E - E[0]).max() / w.n_atoms, "rms max", st[:, 2].max(),
          "T", st[-1, 1])
    assert np.abs(E - E[0]).max() / w.n_atoms < 1e-3
    assert st[:, 2].max() < 1e-3
    assert 100 < st[-1, 1] < 1000
