"""The allocation-free tensor-core product, sxl_mixed_gemm_noalloc.

It serves callers that cannot call cudaMalloc (device memory owned by their
own pool allocator, or already fully reserved): its working storage is a
fixed device array of the library instead of context buffers.  For each
16-bit format (fp16, bf16) and for matrices that fill the array (n = 576)
or only part of it (n = 192, where the tensor maps' row stride is n while
the array's slots are sized for 576), two calls in a row with different
modes and inputs are checked against the context entry point sxl_mixed_gemm
on the same inputs (same kernel and the same order of accumulation, so the
results agree bit for bit; the n = 192 product is compared with the
top-left block of the 576-context product of the zero-padded operands,
whose extra terms are exact zeros) and against the fp64 product within the
bound the other GEMM tests use.  This file is collected last so that a run
stopping at the first failure has run every other test before it; it also
passes on its own in a fresh process (the first call does the per-device
set-up).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_CTX = 576  # 64 atoms: 9 N_at is a multiple of 64, as the context product needs


def _pad(x, n):
    out = np.zeros((2, N_CTX, N_CTX))
    out[:, :n, :n] = x
    return out


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n", [N_CTX, 192])
def test_noalloc_gemm_matches_context_entry_point(prec, n):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl, workload

    ctx = sxl.Context(workload.ModelParams(), N_CTX // 9, [20.0, 20.0, 20.0], prec)
    rng = np.random.default_rng(21 + n)
    cases = [dict(sym=False, split=True, alpha=1.0, beta=0.5, gamma=2.0, with_e=True),
             dict(sym=True, split=False, alpha=-0.5, beta=0.0, gamma=1.0, with_e=False)]
    eps_hi = 2.0 ** -11 if prec == "fp16" else 2.0 ** -8
    eps_split = max(2.0 ** -22 if prec == "fp16" else 2.0 ** -16, 2.0 ** -21)
    for case in cases:
        a = rng.normal(size=(2, n, n)) / np.sqrt(n)
        b = rng.normal(size=(2, n, n)) / np.sqrt(n)
        if case["sym"]:
            b = a  # A A^T is symmetric
        e = rng.normal(size=(2, n, n))
        e = 0.5 * (e + np.transpose(e, (0, 2, 1)))
        A = torch.tensor(a, device="cuda")
        B = torch.tensor(b, device="cuda")
        E = torch.tensor(e, device="cuda") if case["with_e"] else None
        kw = dict(alpha=case["alpha"], beta=case["beta"], gamma=case["gamma"],
                  sym=case["sym"], split=case["split"])
        Ep = torch.tensor(_pad(e, n), device="cuda") if case["with_e"] else None
        ref = ctx.mixed_gemm(torch.tensor(_pad(a, n), device="cuda"),
                             torch.tensor(_pad(b, n), device="cuda"), Ep, **kw)
        ref = ref[:, :n, :n].contiguous()
        out = sxl.mixed_gemm_noalloc(n, prec, A, B, E, **kw)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        exact = case["alpha"] * np.einsum("bij,bkj->bik", a, b) + case["gamma"] * np.eye(n)
        if case["with_e"]:
            exact = exact + case["beta"] * e
        bound = 20 * (eps_split if case["split"] else eps_hi)
        err = np.abs(out.cpu().numpy() - exact).max() / np.abs(exact).max()
        assert err < bound, err
    with pytest.raises(sxl.SxlError):
        z = torch.zeros(2, 640, 640, dtype=torch.float64, device="cuda")
        sxl.mixed_gemm_noalloc(640, prec, z, z)
    ctx.close()
