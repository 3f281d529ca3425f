"""Edge cases on the GPU: the smallest system (a 2-atom dimer, 18 orbitals:
one ragged tile, padded to 64 in the mixed forms) against the oracle, and
calls that do no work."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import electronic, energy  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def sxl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


def _dimer():
    p = wl.ModelParams(krylov_rank=4)
    R = np.array([[0.1, 0.2, 0.3], [2.35, 0.4, 0.1]])   # 2.27 A apart, 6 A box
    cell = np.full(3, 6.0)
    n0 = np.array([0.8, 0.6, -0.9, -0.5])                  # spin-polarized start
    V = np.array([[0.001, 0.0, -0.002], [-0.001, 0.0, 0.002]])
    return p, R, cell, n0, V


@pytest.mark.parametrize("prec", ["fp64", "fp16", "bf16"])
def test_dimer_against_oracle(sxl, prec):
    p, R, cell, n0, _ = _dimer()
    d = electronic.density(R, cell, n0, p)
    ctx = sxl.Context(p, 2, cell, prec)
    q, mu = ctx.density(R, n0)
    tol_q = {"fp64": 1e-10, "fp16": 1e-4, "bf16": 1e-4}[prec]
    assert np.abs(q.cpu().numpy() - d.q).max() < tol_q
    v = wl.random_direction(2, 3)
    qv, _ = ctx.response(v)
    qv_o, _ = d.response(v)
    rel = np.abs(qv.cpu().numpy() - qv_o).max() / np.abs(qv_o).max()
    assert rel < {"fp64": 1e-9, "fp16": 5e-3, "bf16": 5e-2}[prec], rel
    F, en = ctx.forces(R, n0, energies=True)
    tol_f = {"fp64": 1e-8, "fp16": 1e-3, "bf16": 1e-3}[prec]
    assert np.abs(F.cpu().numpy() - energy.forces(d, R, cell)).max() < tol_f
    ctx.close()


def test_zero_step_calls_change_nothing(sxl):
    p, R, cell, n0, V = _dimer()
    ctx = sxl.Context(p, 2, cell, "fp64")
    ctx.set_state(R, V, np.tile(n0, (p.kmax + 1, 1)), float("nan"))
    before = [x.cpu().numpy().copy() for x in ctx.get_state()[:3]]
    ctx.step(0, stats=False)
    ctx.bomd(0, tol=1e-8, mixer="diis", stats=False)
    after = [x.cpu().numpy() for x in ctx.get_state()[:3]]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    cell16 = wl.make_cell(2, seed=3, name="b16")
    b = sxl.Batch([cell16], "fp16")
    b.contexts[0].set_state(cell16.R, cell16.V, np.tile(cell16.n0, (cell16.params.kmax + 1, 1)),
                            float("nan"))
    r0 = b.contexts[0].get_state()[0].cpu().numpy().copy()
    b.step(0)
    assert np.array_equal(b.contexts[0].get_state()[0].cpu().numpy(), r0)
    b.close()
    ctx.close()
