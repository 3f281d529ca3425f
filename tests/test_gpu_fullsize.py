"""Parity at the benchmark's size and configuration: the 1024-atom cell
(9216 orbitals x 2 spins) in the mixed fp16 form, as bench.py runs it,
against the FP64 oracle (dense eigendecomposition) at the neutral start
n = 0 of the benchmark's SCF: charges and spins, one response direction,
the forces and the energies, with the 128-atom tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import electronic, energy, model  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def sxl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


def test_fe1024_fp16_against_oracle(sxl):
    w = wl.fe1024()
    nat = w.n_atoms
    n0 = np.zeros(2 * nat)
    d = electronic.density(w.R, w.cell, n0, w.params)
    ctx = sxl.Context(w.params, nat, w.cell, "fp16", scf_keep_k0=1)
    q, mu = ctx.density(w.R, n0)
    q = q.cpu().numpy()
    err_q = np.abs(q - d.q).max()
    err_m = np.abs((q[:nat] - q[nat:]) - d.spin).max()
    print(f"fe1024 fp16: |dq| {err_q:.2e} |dm| {err_m:.2e} |dmu| {abs(mu - d.mu):.2e}")
    assert err_q < 1e-4 and err_m < 1e-4
    v = wl.random_direction(nat, 21)
    qv, _ = ctx.response(v)
    qv_o, _ = d.response(v)
    rel = np.abs(qv.cpu().numpy() - qv_o).max() / np.abs(qv_o).max()
    bound = ctx.info()["foe_steps"] * 3 * 2.0 ** -12
    print(f"fe1024 fp16: response rel err {rel:.2e} (bound {bound:.2e})")
    assert rel < bound
    F, en = ctx.forces(w.R, n0, energies=True)
    err_f = np.abs(F.cpu().numpy() - energy.forces(d, w.R, w.cell)).max()
    e_o = energy.shadow_energy(d, model.build_h0(w.R, w.cell, w.params),
                               model.repulsive_energy(w.R, w.cell, w.params))
    d_band = abs(en["band"] - e_o["band"]) / nat
    d_u = abs(en["U"] - e_o["U"]) / nat
    print(f"fe1024 fp16: |dF| {err_f:.2e} band/atom {d_band:.2e} U/atom {d_u:.2e}")
    assert err_f < 1e-3
    assert d_band < 1e-4
    assert d_u < 1e-3
    ctx.close()
