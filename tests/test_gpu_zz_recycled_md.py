"""The recycled-subspace kernel (a build choice, not the paper's
construction) in an fp64 trajectory, step by step against the oracle's run
with the same kernel (oracle/dynamics.XLBOMD with recycle=True)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def sxl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


def test_recycled_md_fp64_follows_the_oracle(sxl):
    """40 fp64 sXL-BOMD steps of the 16-atom cell from the SCF point (exact
    K0, rank 4) with the recycled-subspace kernel on both sides (the first
    evaluation by the Krylov construction, then the previous step's
    directions): positions, velocities, n, mu and RMS(q - n) follow the
    oracle's recycled run step by step."""
    from oracle import dynamics
    w = wl.fe16()
    res = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-10)
    md = dynamics.XLBOMD(w.R, w.V, w.cell, res["n"], w.params, res["K0"], mu=res["mu"],
                         recycle=True)
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, "fp64", krylov_recycle=1)
    ctx.set_k0(res["K0"])
    ctx.set_state(w.R, w.V, np.tile(res["n"], (w.params.kmax + 1, 1)), res["mu"])
    for _ in range(40):
        st_o = md.step()
        st = ctx.step(1)[0]
        R, V, nh, mu = ctx.get_state()
        np.testing.assert_allclose(R.cpu().numpy(), md.R, atol=1e-9)
        np.testing.assert_allclose(V.cpu().numpy(), md.V, atol=1e-10)
        np.testing.assert_allclose(nh.cpu().numpy()[0], md.nhist[0], atol=1e-8)
        assert abs(mu - st_o["mu"]) < 1e-8
        assert abs(st[2] - st_o["rms"]) < 1e-8
    ctx.close()
