"""Failure detection, fault injection on the host, checkpoint/resume and the
JSON-lines log, on the GPU.  Nothing here faults, traps or hangs a GPU:

* the bounded-wait self-test waits on a device flag that nothing sets, for
  0.2 s of the global timer, and must come back as SXL_E_TIMEOUT with the
  context still usable;
* faults are injected on the host: NaN positions, a chemical-potential
  search capped at one pass from a far guess, a K0 full of NaN, a corrupted
  or mismatched checkpoint file;
* a checkpoint written after 5 steps and read into a fresh context
  continues the trajectory bit for bit (fp64 at 16 atoms, fp16 at 128)."""
import json
import math
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03529_gb300 import mdlog  # noqa: E402
from paper_2303_03529_gb300 import workload as wl  # noqa: E402


@pytest.fixture(scope="module")
def sxl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl as s
    return s


def _md_context(sxl, w, prec, **kw):
    p = w.params
    ctx = sxl.Context(p, w.n_atoms, w.cell, prec, scf_keep_k0=1, **kw)
    n_star, _, _ = ctx.scf(w.R, np.zeros(ctx.n2), tol=1e-5, max_iter=60)
    _, mu = ctx.density(w.R, n_star)
    ctx.set_state(w.R, w.V, torch.stack([n_star] * (p.kmax + 1)).contiguous(), mu)
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_bounded_wait_times_out_and_context_survives(sxl, prec):
    w = wl.fe16()
    ctx = sxl.Context(w.params, w.n_atoms, w.cell, prec)
    q0, mu0 = ctx.density(w.R, w.n0)
    for _ in range(2):  # the flag is cleared when reported
        t0 = time.perf_counter()
        with pytest.raises(sxl.SxlError) as e:
            ctx.selftest_timeout(0.2)
        dt = time.perf_counter() - t0
        assert e.value.code == sxl.E_TIMEOUT
        assert dt >= 0.19, dt
    q1, mu1 = ctx.density(w.R, w.n0)
    assert torch.equal(q0, q1) and mu0 == mu1
    ctx.close()


def test_host_fault_injection(sxl):
    w = wl.fe16()
    p = w.params
    ctx = sxl.Context(p, w.n_atoms, w.cell, "fp64")
    R_bad = w.R.copy()
    R_bad[3, 1] = np.nan
    with pytest.raises(sxl.SxlError) as e:
        ctx.density(R_bad, w.n0)
    assert e.value.code == sxl.E_NAN
    q, mu = ctx.density(w.R, w.n0)  # usable again
    assert np.isfinite(q.cpu().numpy()).all()
    capped = sxl.Context(p, w.n_atoms, w.cell, "fp64", mu_max_iter=1)
    with pytest.raises(sxl.SxlError) as e:
        capped.density(w.R, w.n0, mu + 3.0)
    assert e.value.code == sxl.E_NO_CONVERGENCE
    capped.close()
    # a K0 of NaN: the next step's n is not finite, which the density reports
    ctx.set_state(w.R, w.V, np.tile(w.n0, (p.kmax + 1, 1)), mu)
    ctx.set_k0(np.full((ctx.n2, ctx.n2), np.nan))
    with pytest.raises(sxl.SxlError) as e:
        ctx.step(3, stats=False)
    assert e.value.code == sxl.E_NAN
    ctx.set_k0()
    ctx.set_state(w.R, w.V, np.tile(w.n0, (p.kmax + 1, 1)), mu)
    st = ctx.step(2)
    assert np.isfinite(st).all()
    ctx.close()


@pytest.mark.parametrize("prec,wname", [("fp64", "fe16"), ("fp16", "fe128")])
def test_checkpoint_resume_is_bit_identical(sxl, tmp_path, prec, wname):
    w = getattr(wl, wname)()
    a = _md_context(sxl, w, prec)
    a.step(5, stats=False)
    path = str(tmp_path / "state.ckpt")
    a.checkpoint_write(path)
    st_a = a.step(5)
    Ra, Va, nha, mua = a.get_state()
    assert a.md_step() == 10
    b = sxl.Context(w.params, w.n_atoms, w.cell, prec, scf_keep_k0=1)
    b.checkpoint_read(path)
    assert b.md_step() == 5
    st_b = b.step(5)
    Rb, Vb, nhb, mub = b.get_state()
    print(f"{prec} {wname}: resumed E_tot {st_b[-1, 0]:.10f} vs {st_a[-1, 0]:.10f}")
    assert torch.equal(Ra, Rb) and torch.equal(Va, Vb) and torch.equal(nha, nhb)
    assert mua == mub
    assert np.array_equal(st_a, st_b)
    assert b.md_step() == 10
    a.close()
    b.close()


def test_checkpoint_rejects_bad_files(sxl, tmp_path):
    w = wl.fe16()
    a = _md_context(sxl, w, "fp64")
    a.step(2, stats=False)
    path = tmp_path / "state.ckpt"
    a.checkpoint_write(str(path))
    raw = bytearray(path.read_bytes())
    raw[-9] ^= 0x40  # one bit of the payload (K0)
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    R0, V0, nh0, mu0 = a.get_state()
    with pytest.raises(sxl.SxlError) as e:
        a.checkpoint_read(str(bad))
    assert e.value.code == sxl.E_IO
    R1, V1, nh1, mu1 = a.get_state()  # left as it was
    assert torch.equal(R0, R1) and torch.equal(nh0, nh1) and mu0 == mu1
    w128 = wl.fe128()
    other = sxl.Context(w128.params, w128.n_atoms, w128.cell, "fp64")
    with pytest.raises(sxl.SxlError) as e:
        other.checkpoint_read(str(path))
    assert e.value.code == sxl.E_IO
    with pytest.raises(sxl.SxlError) as e:
        other.checkpoint_read(str(tmp_path / "missing.ckpt"))
    assert e.value.code == sxl.E_IO
    other.close()
    a.close()


def test_jsonl_log_of_a_run(sxl, tmp_path):
    w = wl.fe16()
    ctx = _md_context(sxl, w, "fp16")
    path = tmp_path / "md.jsonl"
    recs = mdlog.run(ctx, 6, path, every=3)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines == recs and [r["step"] for r in lines] == [3, 6]
    for r in lines:
        assert math.isfinite(r["E_tot_per_atom"]) and r["T"] > 0 and r["rms_q_minus_n"] < 1e-2
        assert math.isfinite(r["m_total"]) and r["wall_s_per_step"] > 0
    ctx.close()


def test_checkpoint_format_shared_with_the_host_reader(sxl, tmp_path):
    """A checkpoint the library writes reads back on the host with the same
    arrays (paper_2303_03529_gb300.checkpoint); one the host writes from
    them, with a new step counter, reads into a fresh context and continues
    like the original."""
    from paper_2303_03529_gb300 import checkpoint
    w = wl.fe16()
    a = _md_context(sxl, w, "fp64")
    a.step(3, stats=False)
    p1 = tmp_path / "lib.ckpt"
    a.checkpoint_write(str(p1))
    ck = checkpoint.read(p1)
    R, V, nh, mu = a.get_state()
    assert ck["md_step"] == 3 and ck["mu"] == mu and ck["n_atoms"] == w.n_atoms
    np.testing.assert_array_equal(ck["R"], R.cpu().numpy())
    np.testing.assert_array_equal(ck["V"], V.cpu().numpy())
    np.testing.assert_array_equal(ck["nhist"], nh.cpu().numpy())
    p2 = tmp_path / "host.ckpt"
    checkpoint.write(p2, dict(ck, md_step=100))
    b = sxl.Context(w.params, w.n_atoms, w.cell, "fp64", scf_keep_k0=1)
    b.checkpoint_read(str(p2))
    assert b.md_step() == 100
    st_a, st_b = a.step(2), b.step(2)
    assert np.array_equal(st_a, st_b)
    a.close()
    b.close()
