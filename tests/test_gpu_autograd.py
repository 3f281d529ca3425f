"""Differentiation form: the shadow energy as a torch.autograd.Function whose
backward is the library's force kernel (adjoint of U with respect to R at
constant n).  Checked against Richardson-extrapolated central differences of
U (h = 2e-3 and 1e-3 A, truncation O(h^4)) on seeded coordinates and against
the oracle gradient."""
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


@pytest.mark.parametrize("which", ["fe16", "cell54"])
def test_autograd_gradient_fd_and_oracle(sxl, which):
    w = wl.fe16() if which == "fe16" else wl.make_cell(3, seed=54, name="cell54")
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, "fp64")
    R = torch.tensor(w.R, device="cuda", requires_grad=True)
    n = torch.tensor(w.n0, device="cuda")
    U = sxl.shadow_energy(R, n, ctx)
    U.backward()
    g = R.grad.detach().cpu().numpy()
    # oracle gradient dU/dR = -F_oracle
    d = electronic.density(w.R, w.cell, w.n0, w.params)
    np.testing.assert_allclose(g, -energy.forces(d, w.R, w.cell), atol=1e-8)
    # central differences of the GPU energy on seeded coordinates
    rng = np.random.default_rng(20)

    def central(a, c, h):
        Rp = w.R.copy()
        Rp[a, c] += h
        Rm = w.R.copy()
        Rm[a, c] -= h
        up = sxl.shadow_energy(torch.tensor(Rp, device="cuda"), n, ctx).item()
        um = sxl.shadow_energy(torch.tensor(Rm, device="cuda"), n, ctx).item()
        return (up - um) / (2 * h)

    for _ in range(6):
        a, c = int(rng.integers(w.n_atoms)), int(rng.integers(3))
        d1, d2 = central(a, c, 2e-3), central(a, c, 1e-3)
        assert abs((4 * d2 - d1) / 3 - g[a, c]) < 1e-7
    ctx.close()


def test_autograd_mixed_vs_oracle(sxl):
    """fp16 form at 128 atoms: the gradient matches the oracle within the
    mixed-form force tolerance (1e-3 eV/A)."""
    w = wl.fe128()
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, "fp16")
    R = torch.tensor(w.R, device="cuda", requires_grad=True)
    n = torch.tensor(w.n0, device="cuda")
    sxl.shadow_energy(R, n, ctx).backward()
    d = electronic.density(w.R, w.cell, w.n0, w.params)
    err = np.abs(R.grad.cpu().numpy() + energy.forces(d, w.R, w.cell)).max()
    assert err < 1e-3, err
    ctx.close()
