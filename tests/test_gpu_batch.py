"""Batched replicas: independent cells of different sizes (padded chains
included) stepped together on their own streams from a pool of host
threads.  A batched step gives the same state, bit for bit, as stepping each
replica alone; one replica's sXL-BOMD steps follow the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dynamics  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def sxl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


def _cells():
    return [wl.make_cell(3, seed=7001, sigma=0.05, name="r54"),
            wl.make_cell(4, seed=7002, sigma=0.08, vacancy_frac=0.03, name="r124"),
            wl.make_cell(5, seed=7003, sigma=0.04, name="r250")]


def _state(ctx, w):
    nat = w.R.shape[0]
    ctx.set_state(w.R, w.V, np.tile(w.n0, (w.params.kmax + 1, 1)), float("nan"))


def test_batch_equals_solo(sxl):
    cells = _cells()
    solo = []
    for w in cells:
        ctx = sxl.Context(w.params, w.R.shape[0], w.cell, "fp16")
        _state(ctx, w)
        ctx.step(2, stats=False)
        R, V, nh, mu = ctx.get_state()
        solo.append((R.cpu().numpy(), V.cpu().numpy(), nh.cpu().numpy(), mu))
        ctx.close()
    b = sxl.Batch(cells, "fp16")
    for ctx, w in zip(b.contexts, cells):
        _state(ctx, w)
    status = b.step(2, nthreads=3)
    assert (status == 0).all()
    for ctx, ref in zip(b.contexts, solo):
        R, V, nh, mu = ctx.get_state()
        assert np.array_equal(R.cpu().numpy(), ref[0])
        assert np.array_equal(V.cpu().numpy(), ref[1])
        assert np.array_equal(nh.cpu().numpy(), ref[2])
        assert mu == ref[3]
    b.close()


def test_batch_replica_follows_oracle(sxl):
    """The 54-atom replica (padded chain, fp16) against the oracle's
    XL-BOMD with the same K0 = -I, two steps from the oracle's SCF fixed
    point (the state MD starts from): positions to 1e-6 A, velocities to
    1e-5 A/fs and n to 1e-4 e (the mixed form's force and charge errors are
    about 1e-4 eV/A and 1e-5 e)."""
    cells = _cells()
    w = cells[0]
    nat = w.R.shape[0]
    n_star = dynamics.scf(w.R, w.cell, w.n0, w.params, tol=1e-9)["n"]
    b = sxl.Batch(cells, "fp16")
    for ctx, c in zip(b.contexts, cells):
        _state(ctx, c)
    b.contexts[0].set_state(w.R, w.V, np.tile(n_star, (w.params.kmax + 1, 1)), float("nan"))
    md = dynamics.XLBOMD(w.R, w.V, w.cell, n_star, w.params, -np.eye(2 * nat))
    for _ in range(2):
        md.step()
        b.step(1)
    R, V, nh, mu = b.contexts[0].get_state()
    np.testing.assert_allclose(R.cpu().numpy(), md.R, atol=1e-6)
    np.testing.assert_allclose(V.cpu().numpy(), md.V, atol=1e-5)
    np.testing.assert_allclose(nh.cpu().numpy()[0], md.nhist[0], atol=1e-4)
    b.close()
