"""The paper-general model at the benchmark's size (1024 atoms, 9216
orbitals x 2 spins, overlap and shell-resolved charges and spins) in each
mixed form, at the cell's start (n = 0 per shell), against the general
oracle (generalized eigenproblem at 9216 orbitals, about two minutes on the
host in a spawned worker).

Checked: the shell charges and spins (1e-4 e), the forces with the overlap
terms (1e-3 eV/A) and the shadow energy (1e-3 eV/atom fp16, 5e-3 bf16).
bf16 pairs carry about 2^-18 of each chain product, which puts the spins at
about 1.1e-4 e here: the test records that as an expected failure after the
other checks, and fails if it grows past 2e-4."""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03529_gb300 import workload as wl  # noqa: E402


def _oracle_eval():
    from oracle import general, model
    w = wl.fe1024_general()
    d = general.density(w.R, w.cell, w.n0, w.params)
    F = general.forces(d, w.R, w.cell)
    U = general.shadow_energy(d, model.build_h0(w.R, w.cell, w.params),
                              model.repulsive_energy(w.R, w.cell, w.params))["U"]
    return d.q, d.spin, d.mu, F, U


@pytest.fixture(scope="module")
def oracle_future():
    ex = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
    fut = ex.submit(_oracle_eval)
    yield fut
    ex.shutdown()


@pytest.fixture(scope="module")
def sxl(oracle_future):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_fe1024_general_mixed_against_oracle(sxl, oracle_future, prec):
    w = wl.fe1024_general()
    p, nat = w.params, w.n_atoms
    ctx = sxl.Context(p, nat, w.cell, prec)
    q, mu = ctx.density(w.R, w.n0)
    F, en = ctx.forces(w.R, w.n0, energies=True)
    q, F, U = q.cpu().numpy(), F.cpu().numpy(), en["U"]
    ctx.close()
    q_o, m_o, mu_o, F_o, U_o = oracle_future.result()
    G = 3 * nat
    err_q = np.abs(q - q_o).max()
    err_m = np.abs((q[:G] - q[G:]) - m_o).max()
    err_f = np.abs(F - F_o).max()
    err_u = abs(U - U_o) / nat
    print(f"fe1024_general {prec}: |dq| {err_q:.2e} |dm| {err_m:.2e} |dmu| {abs(mu - mu_o):.2e} "
          f"|dF| {err_f:.2e} dU/atom {err_u:.2e}")
    assert err_f < 1e-3
    assert err_u < (1e-3 if prec == "fp16" else 5e-3)
    if prec == "bf16":
        assert err_q < 2e-4 and err_m < 2e-4
        if err_q >= 1e-4 or err_m >= 1e-4:
            pytest.xfail(f"bf16 general model at 1024 atoms: |dq| {err_q:.2e}, |dm| {err_m:.2e} "
                         "above 1e-4 e")
    assert err_q < 1e-4 and err_m < 1e-4
