"""Mixed-precision (tcgen05, fp16 / bf16 with fp32 accumulation) path.

1. The tensor-core GEMM against an fp64 product of the same inputs, at
   N = 1152 (9 row tiles of 128, 4.5 column tiles of 256: a ragged edge),
   in plain, split, symmetric and epilogue (beta E + gamma I) modes.  Bounds
   follow from the arithmetic: inputs rounded to hi (fp16: 2^-11, bf16: 2^-8
   relative) for the plain form, hi + lo 2^-12 for the split form, fp32
   accumulation over K = 1152 terms.
2. The mixed density (q, mu), response q_v, forces and shadow energy at
   128 atoms against the FP64 oracle, with the tolerances of the mixed form
   in both 16-bit formats: 1e-4 e on charges and spins and 1e-3 eV/A on
   forces; band energy 1e-4 eV/atom (fp16) and 1e-3 (bf16), total shadow
   energy (with the entropy) 1e-3 eV/atom (fp16) and 5e-3 (bf16), whose
   16-bit pairs carry about 16 significant bits against fp16's 22.
"""
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


def _sym(rng, n, scale=1.0):
    a = rng.normal(size=(n, n)) * scale / np.sqrt(n)
    return 0.5 * (a + a.T)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_gemm_against_fp64(sxl, prec):
    w = wl.fe128()
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, prec)
    n = w.n_orb
    rng = np.random.default_rng(0)
    A = np.stack([_sym(rng, n), _sym(rng, n)])
    B = np.stack([_sym(rng, n), _sym(rng, n)])
    E = np.stack([_sym(rng, n), _sym(rng, n)])
    ref = np.einsum("bij,bkj->bik", A, B)
    eps_hi = 2.0 ** -11 if prec == "fp16" else 2.0 ** -8
    eps_split = 2.0 ** -22 if prec == "fp16" else 2.0 ** -16
    scale = np.abs(ref).max()
    # plain: hi x hi
    C = ctx.mixed_gemm(A, B, split=False).cpu().numpy()
    err = np.abs(C - ref).max() / scale
    assert err < 20 * eps_hi, err
    # split: hi x hi + (hi x lo + lo x hi) 2^-12
    C = ctx.mixed_gemm(A, B, split=True).cpu().numpy()
    err = np.abs(C - ref).max() / scale
    assert err < 20 * max(eps_split, 2.0 ** -21), err
    # symmetric product with epilogue: 0.5 A A^T - 2 E + 3 I, mirrored tiles
    ref2 = 0.5 * np.einsum("bij,bkj->bik", A, A) - 2.0 * E + 3.0 * np.eye(n)
    C = ctx.mixed_gemm(A, A, E, alpha=0.5, beta=-2.0, gamma=3.0, sym=True, split=True)
    C = C.cpu().numpy()
    np.testing.assert_array_equal(C, np.transpose(C, (0, 2, 1)))
    err = np.abs(C - ref2).max() / np.abs(ref2).max()
    assert err < 20 * max(eps_split, 2.0 ** -21), err
    ctx.close()


def _response_bound(ctx, prec):
    """The response products run on the hi parts alone: each chain step
    rounds three operands to hi (half an ulp: 2^-12 fp16, 2^-9 bf16), and a
    relative error entering at step k keeps its size through the later
    doublings, so the bound is n_r * 3 * 2^-12 (fp16) or 2^-9 (bf16)."""
    u = 2.0 ** -12 if prec == "fp16" else 2.0 ** -9
    return ctx.info()["foe_steps"] * 3 * u


@pytest.fixture(scope="module")
def dens128():
    w = wl.fe128()
    return w, electronic.density(w.R, w.cell, w.n0, w.params)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_mixed_density_and_response(sxl, dens128, prec):
    w, d = dens128
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, prec)
    q, mu = ctx.density(w.R, w.n0)
    q = q.cpu().numpy()
    err_q = np.abs(q - d.q).max()
    err_m = np.abs((q[:128] - q[128:]) - d.spin).max()
    print(f"{prec}: |dq| {err_q:.2e} |dm| {err_m:.2e} |dmu| {abs(mu - d.mu):.2e}")
    assert err_q < 1e-4 and err_m < 1e-4
    v = wl.random_direction(128, 11)
    qv, _ = ctx.response(v)
    qv_o, _ = d.response(v)
    rel = np.abs(qv.cpu().numpy() - qv_o).max() / np.abs(qv_o).max()
    print(f"{prec}: response rel err {rel:.2e}")
    assert rel < _response_bound(ctx, prec)
    F, en = ctx.forces(w.R, w.n0, energies=True)
    err_f = np.abs(F.cpu().numpy() - energy.forces(d, w.R, w.cell)).max()
    print(f"{prec}: |dF| {err_f:.2e}")
    assert err_f < 1e-3
    from oracle import model
    e_o = energy.shadow_energy(d, model.build_h0(w.R, w.cell, w.params),
                               model.repulsive_energy(w.R, w.cell, w.params))
    per_atom = {k: abs(en[k] - e_o[k]) / w.n_atoms for k in ("U", "band", "entropy")}
    print(f"{prec}: energy errors per atom {per_atom}")
    # band energy follows D; the entropy is a small difference of traces of
    # size sum |y| (~4.6e4 per spin here), so a relative error of ~1e-5 in
    # the 16-bit-pair chain shows up as ~4e-4 eV/atom
    assert per_atom["band"] < (1e-4 if prec == "fp16" else 1e-3)
    assert per_atom["U"] < (1e-3 if prec == "fp16" else 5e-3)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("ncell,vac", [(3, 0.0), (2, 0.0), (3, 0.04)])
def test_mixed_padded_chain(sxl, prec, ncell, vac):
    """Cells whose 9 N_at is not a multiple of 64 (54 atoms: N = 486 -> 512;
    16 atoms: 144 -> 192; 52 atoms with vacancies: 468 -> 512) run the
    chain on the padded dimension; q, m, the response, the forces and the
    shadow energy match the FP64 oracle with the 128-atom tolerances."""
    w = wl.make_cell(ncell, seed=5400 + ncell, sigma=0.06, vacancy_frac=vac, name="padded")
    nat = w.R.shape[0]
    assert (9 * nat) % 64 != 0
    d = electronic.density(w.R, w.cell, w.n0, w.params)
    ctx = sxl.Context(w.params, nat, w.cell, prec)
    q, mu = ctx.density(w.R, w.n0)
    q = q.cpu().numpy()
    err_q = np.abs(q - d.q).max()
    err_m = np.abs((q[:nat] - q[nat:]) - d.spin).max()
    print(f"padded {nat} {prec}: |dq| {err_q:.2e} |dm| {err_m:.2e} |dmu| {abs(mu - d.mu):.2e}")
    assert err_q < 1e-4 and err_m < 1e-4
    v = wl.random_direction(nat, 12)
    qv, _ = ctx.response(v)
    qv_o, _ = d.response(v)
    rel = np.abs(qv.cpu().numpy() - qv_o).max() / np.abs(qv_o).max()
    assert rel < _response_bound(ctx, prec), rel
    F, en = ctx.forces(w.R, w.n0, energies=True)
    err_f = np.abs(F.cpu().numpy() - energy.forces(d, w.R, w.cell)).max()
    assert err_f < 1e-3, err_f
    from oracle import model
    e_o = energy.shadow_energy(d, model.build_h0(w.R, w.cell, w.params),
                               model.repulsive_energy(w.R, w.cell, w.params))
    dU = abs(en["U"] - e_o["U"]) / nat
    print(f"padded {nat} {prec}: rel {rel:.2e} |dF| {err_f:.2e} dU/atom {dU:.2e}")
    assert dU < (1e-3 if prec == "fp16" else 5e-3)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_every_tile_choice_gives_the_product(sxl, prec):
    """Every tile the autotuner may pick (plain: K block 64/32 x 256/128-row
    tiles or the persistent kernel; split: K block 32/64; dual: 256/128-row
    tiles or the persistent kernel) computes the same
    product within the form's bound at N = 1152 (ragged 256-column edge), and
    the autotuner returns one of them."""
    w = wl.fe128()
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, prec)
    n = w.n_orb
    rng = np.random.default_rng(3)
    A = np.stack([_sym(rng, n), _sym(rng, n)])
    B = np.stack([_sym(rng, n), _sym(rng, n)])
    ref = np.einsum("bij,bkj->bik", A, B)
    ref_dual = ref + np.einsum("bij,bkj->bik", B, A)
    eps_hi = 2.0 ** -11 if prec == "fp16" else 2.0 ** -8
    eps_split = max(2.0 ** -22 if prec == "fp16" else 2.0 ** -16, 2.0 ** -21)
    for bk in (64, 32):
        for mt in (2, 1):
            ctx.set_tiles(bk_plain=bk, mt_plain=mt, bk_split=bk, mt_dual=mt)
            C = ctx.mixed_gemm(A, B, split=False).cpu().numpy()
            assert np.abs(C - ref).max() / np.abs(ref).max() < 20 * eps_hi, (bk, mt)
            C = ctx.mixed_gemm(A, B, split=True).cpu().numpy()
            assert np.abs(C - ref).max() / np.abs(ref).max() < 20 * eps_split, (bk, mt)
            C = ctx.mixed_gemm(A, B, sym=True, split=2).cpu().numpy()
            assert np.abs(C - ref_dual).max() / np.abs(ref_dual).max() < 40 * eps_hi, (bk, mt)
    ctx.set_product_kernel("persistent")
    C = ctx.mixed_gemm(A, B, split=False).cpu().numpy()
    assert np.abs(C - ref).max() / np.abs(ref).max() < 20 * eps_hi
    C = ctx.mixed_gemm(A, B, sym=True, split=2).cpu().numpy()
    assert np.abs(C - ref_dual).max() / np.abs(ref_dual).max() < 40 * eps_hi
    ctx.set_product_kernel("default")
    t = ctx.autotune()
    print(f"{prec} autotune at N = {n}: {t}")
    assert t["plain_bk"] in (32, 64) and t["plain_rows"] in (128, 256)
    assert t["split_bk"] in (32, 64) and t["dual_rows"] in (128, 256)
    assert isinstance(t["plain_persistent"], bool) and isinstance(t["dual_persistent"], bool)
    with pytest.raises(sxl.SxlError):
        ctx.set_tiles(bk_plain=48)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n", [576, 1152, 2304])
def test_persistent_products_match(sxl, prec, n):
    """The persistent plain/dual kernel (256 x 128 tiles walked by one CTA
    per SM, two TMEM accumulator stages) against fp64 and against the
    single-tile kernel: plain C = A B^T, the symmetric A A^T with E and
    gamma I, and the dual A B^T + B A^T (symmetric).  N = 576 and 2304 leave
    partial 256-row tiles and an uneven number of tiles per CTA; each output
    element sums the same k steps in the same order in both kernels."""
    ctx = sxl.Context(wl.ModelParams(), n // 9, [60.0, 60.0, 60.0], prec)
    rng = np.random.default_rng(7)
    A = np.stack([_sym(rng, n), _sym(rng, n)])
    B = np.stack([_sym(rng, n), _sym(rng, n)])
    E = np.stack([_sym(rng, n), _sym(rng, n)])
    ref = np.einsum("bij,bkj->bik", A, B)
    ref_sym = 0.5 * np.einsum("bij,bkj->bik", A, A) + 0.25 * E + 0.75 * np.eye(n)
    ref_dual = ref + np.einsum("bij,bkj->bik", B, A)
    eps_hi = 2.0 ** -11 if prec == "fp16" else 2.0 ** -8
    out = {}
    for kern in ("persistent", "single"):
        ctx.set_product_kernel(kern)
        C = ctx.mixed_gemm(A, B, split=False).cpu().numpy()
        Cs = ctx.mixed_gemm(A, A, E=E, alpha=0.5, beta=0.25, gamma=0.75, sym=True,
                            split=False).cpu().numpy()
        Cd = ctx.mixed_gemm(A, B, sym=True, split=2).cpu().numpy()
        assert np.abs(C - ref).max() / np.abs(ref).max() < 20 * eps_hi, kern
        assert np.abs(Cs - ref_sym).max() / np.abs(ref_sym).max() < 20 * eps_hi, kern
        assert np.abs(Cs - Cs.transpose(0, 2, 1)).max() == 0.0, kern
        assert np.abs(Cd - ref_dual).max() / np.abs(ref_dual).max() < 40 * eps_hi, kern
        out[kern] = (C, Cs, Cd)
    for a, b, what in zip(out["persistent"], out["single"], ("plain", "sym", "dual")):
        d = np.abs(a - b).max()
        print(f"{prec} n {n} {what}: persistent vs single-tile max diff {d:.3e}")
        assert d <= 1e-6 * np.abs(b).max(), what
    ctx.close()



@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tuned_k_block_keeps_the_k_halves(sxl, prec):
    """The density chain's split products run as two launches over K halves.
    A context whose split K block differs from the library default (64
    against 32) must count those halves in its own block width: the same
    density within the form's noise, and the same tensor-core work (a
    mis-counted range covered all of K in the first launch and again, as
    zeros, in the second)."""
    w = wl.fe128()
    out = {}
    for bk in (32, 64):
        ctx = sxl.Context(w.params, w.n_atoms, w.cell, prec)
        ctx.set_tiles(bk_split=bk)
        ctx.enable_gemm_timing(True)
        q, mu = ctx.density(w.R, w.n0)
        t = ctx.gemm_timers(reset=True)["split"]
        out[bk] = (q.cpu().numpy(), mu, t["issued_flops"] / max(t["launches"], 1))
        ctx.close()
    dq = np.abs(out[32][0] - out[64][0]).max()
    print(f"{prec}: K block 32 vs 64: |dq| {dq:.2e}, issued flops per launch "
          f"{out[32][2]:.4e} / {out[64][2]:.4e}")
    assert dq < 5e-5
    assert abs(out[64][2] / out[32][2] - 1.0) < 1e-12


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n", [576, 1152])
def test_fused_products_match_unfused(sxl, prec, n):
    """The fused products of m right-hand sides (one persistent launch over
    2 m matrices, operands shared across the right-hand sides or not) give,
    block by block, the unfused products bit for bit: the plain form with a
    shared left operand (the response chain's V = A+ dT), the dual symmetric
    form with a shared right operand and an E term (the chain's start, dQ)
    and with a shared left operand (the chain's A- V^T + V A-)."""
    m = 3
    ctx = sxl.Context(wl.ModelParams(), n // 9, [60.0, 60.0, 60.0], prec)
    rng = np.random.default_rng(5)
    sh = np.stack([_sym(rng, n), _sym(rng, n)])                     # one per spin
    per = np.stack([_sym(rng, n) for _ in range(2 * m)])            # one per (j, spin)
    E = np.stack([_sym(rng, n) for _ in range(2 * m)])
    cases = [
        dict(X=sh, x_per=False, Y=per, y_per=True, sym=False, dual=False, E=None),
        dict(X=per, x_per=True, Y=sh, y_per=False, sym=True, dual=True, E=E),
        dict(X=sh, x_per=False, Y=per, y_per=True, sym=True, dual=True, E=None),
    ]
    for k, cs in enumerate(cases):
        C = ctx.mixed_gemm_fused(cs["X"], cs["Y"], m, cs["x_per"], cs["y_per"], E=cs["E"],
                                 alpha=0.5, beta=0.25 if cs["E"] is not None else 0.0, gamma=0.75,
                                 sym=cs["sym"], dual=cs["dual"]).cpu().numpy()
        for j in range(m):
            Xj = cs["X"][2 * j:2 * j + 2] if cs["x_per"] else cs["X"]
            Yj = cs["Y"][2 * j:2 * j + 2] if cs["y_per"] else cs["Y"]
            Ej = cs["E"][2 * j:2 * j + 2] if cs["E"] is not None else None
            ref = ctx.mixed_gemm(Xj, Yj, E=Ej, alpha=0.5, beta=0.25 if Ej is not None else 0.0,
                                 gamma=0.75, sym=cs["sym"], split=2 if cs["dual"] else 0).cpu().numpy()
            d = np.abs(C[2 * j:2 * j + 2] - ref).max()
            assert d == 0.0, (k, j, d)
    ctx.close()
