"""Pins of the oracle's model (Sec. III.A): the Slater-Koster table, the
smooth cutoff, the periodic image sum and the Coulomb matrix.

None of these re-types an oracle formula: the SK table is checked through
rotational covariance (with the d-orbital rotation fitted numerically from
the orbital shapes) and its canonical form on the z axis; the image sum
through band folding into a larger supercell."""
import numpy as np
import pytest

from oracle import model
from paper_2303_03529_gb300 import workload as wl

P = wl.ModelParams()


def _orbital_shapes(pts):
    """Real angular shapes with equal sphere norm: s, x, y, z, sqrt3 xy,
    sqrt3 yz, sqrt3 zx, sqrt3/2 (x2 - y2), z2 - (x2 + y2)/2."""
    x, y, z = pts.T
    s3 = np.sqrt(3.0)
    return np.stack([np.ones_like(x), x, y, z, s3 * x * y, s3 * y * z, s3 * z * x,
                     0.5 * s3 * (x * x - y * y), z * z - 0.5 * (x * x + y * y)], axis=1)


def _orbital_rotation(Q, rng):
    """O with phi_a(Q^T r) = sum_c O[c, a] phi_c(r), by least squares on
    random points (exact, since each l-shell is rotation invariant)."""
    pts = rng.normal(size=(200, 3))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    A = _orbital_shapes(pts)
    B = _orbital_shapes(pts @ Q)   # rows: phi(Q^T r) for r = pts
    O = np.zeros((9, 9))
    for blk in (slice(0, 1), slice(1, 4), slice(4, 9)):
        sol = np.linalg.lstsq(A[:, blk], B[:, blk], rcond=None)[0]
        O[blk, blk] = sol
    return O


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_sk_canonical_z_axis():
    r = 2.7
    E = model.sk_block(np.array([0.0, 0.0, r]), P)
    V = model.bond_integrals(r, P)
    sss, sps, sds, pps, ppp, pds, pdp, dds, ddp, ddd = V
    s, x, y, z, xy, yz, zx, x2, z2 = range(9)
    expect = np.zeros((9, 9))
    expect[s, s] = sss
    expect[s, z] = sps
    expect[z, s] = -sps
    expect[s, z2] = sds
    expect[z2, s] = sds
    expect[z, z] = pps
    expect[x, x] = expect[y, y] = ppp
    expect[z, z2] = pds
    expect[z2, z] = -pds
    expect[x, zx] = expect[y, yz] = pdp
    expect[zx, x] = expect[yz, y] = -pdp
    expect[z2, z2] = dds
    expect[yz, yz] = expect[zx, zx] = ddp
    expect[xy, xy] = expect[x2, x2] = ddd
    np.testing.assert_allclose(E, expect, atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_sk_rotational_covariance(seed):
    """E(Q d) = O E(d) O^T for the orbital rotation O of Q: pins every entry."""
    rng = np.random.default_rng(100 + seed)
    Q = _random_rotation(rng)
    O = _orbital_rotation(Q, rng)
    np.testing.assert_allclose(O @ O.T, np.eye(9), atol=1e-12)
    for r in (2.3, 2.9, 4.7):
        d = np.array([0.0, 0.0, r])
        E0 = model.sk_block(d, P)
        E1 = model.sk_block(Q @ d, P)
        np.testing.assert_allclose(E1, O @ E0 @ O.T, atol=1e-12)


def test_sk_inversion_parity():
    rng = np.random.default_rng(7)
    d = rng.normal(size=3) * 1.5
    E = model.sk_block(d, P)
    Em = model.sk_block(-d, P)
    np.testing.assert_allclose(Em, E.T, atol=1e-14)


def test_switch_is_c2():
    f = lambda r: model.switch(r, P.r_on, P.r_cut)
    h = 1e-5
    for r0, val in ((P.r_on, 1.0), (P.r_cut, 0.0)):
        assert abs(f(r0) - val) < 1e-15
        # one-sided first and second derivatives vanish on both sides
        for sgn in (-1, 1):
            d1 = (f(r0 + sgn * h) - f(r0)) / (sgn * h)
            d2 = (f(r0 + 2 * sgn * h) - 2 * f(r0 + sgn * h) + f(r0)) / (h * h)
            assert abs(d1) < 1e-8
            assert abs(d2) < 2e-2   # a C1-only switch would give |f''| ~ 24 here
    rr = np.linspace(P.r_on, P.r_cut, 50)
    vals = np.array([f(r) for r in rr])
    assert np.all(np.diff(vals) <= 1e-15)


def test_h0_image_sum_band_folding():
    """Gamma-point eigenvalues of a 2x2x2 cell (L < 2 r_cut, images summed)
    are a subset of those of the same arrangement repeated 2x2x2 times."""
    w = wl.make_cell(2, seed=11, sigma=0.05)
    H_small = model.build_h0(w.R, w.cell, P)
    L = w.cell
    reps = [w.R + np.array([i, j, k]) * L for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    H_big = model.build_h0(np.concatenate(reps), 2 * L, P)
    ev_s = np.linalg.eigvalsh(H_small)
    ev_b = np.linalg.eigvalsh(H_big)
    for e in ev_s:
        assert np.min(np.abs(ev_b - e)) < 1e-10
    np.testing.assert_allclose(H_small, H_small.T, atol=1e-15)


def test_h0_dimer_block():
    R = np.array([[1.0, 1.0, 1.0], [2.5, 2.2, 1.9]])
    cell = np.array([30.0, 30.0, 30.0])
    H = model.build_h0(R, cell, P)
    np.testing.assert_allclose(H[:9, 9:], model.sk_block(R[1] - R[0], P), atol=1e-15)
    np.testing.assert_allclose(np.diag(H[:9, :9]), model.onsite(P))


def test_gamma_matrix():
    w = wl.make_cell(3, seed=3)
    G = model.gamma_matrix(w.R, w.cell, P)
    np.testing.assert_allclose(G, G.T, atol=1e-15)
    np.testing.assert_allclose(np.diag(G), P.U)
    # far pair in a big box: tends to k / r
    R = np.array([[0.0, 0, 0], [40.0, 0, 0]])
    G2 = model.gamma_matrix(R, np.array([200.0, 200, 200]), P)
    assert abs(G2[0, 1] - P.coulomb_k / 40.0) < 1e-6
