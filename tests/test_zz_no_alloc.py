"""The allocation-free tensor-core product, sxl_mixed_gemm_noalloc.

It serves callers that cannot call cudaMalloc (device memory owned by their
own pool allocator, or already fully reserved): its working storage is a
fixed device array of the library instead of context buffers.  Two calls in
a row, with different modes and inputs, are checked against the context
entry point sxl_mixed_gemm on the same inputs (same kernel, so the results
must agree bit for bit) and against the fp64 product within the split-form
bound the other GEMM tests use.  This file is collected last so that a run
stopping at the first failure has run every other test before it; it also
passes on its own in a fresh process (the first call does the per-device
set-up).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_gemm_matches_context_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03529_gb300 import sxl, workload

    n_atoms, n = 64, 576
    ctx = sxl.Context(workload.ModelParams(), n_atoms, [20.0, 20.0, 20.0], "fp16")
    rng = np.random.default_rng(21)
    cases = [dict(sym=False, split=True, alpha=1.0, beta=0.5, gamma=2.0, with_e=True),
             dict(sym=True, split=False, alpha=-0.5, beta=0.0, gamma=1.0, with_e=False)]
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
        ref = ctx.mixed_gemm(A, B, E, **kw)
        out = sxl.mixed_gemm_noalloc(n, "fp16", A, B, E, **kw)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        exact = case["alpha"] * np.einsum("bij,bkj->bik", a, b) + case["gamma"] * np.eye(n)
        if case["with_e"]:
            exact = exact + case["beta"] * e
        bound = 20 * (2.0 ** -21 if case["split"] else 2.0 ** -11)
        err = np.abs(out.cpu().numpy() - exact).max() / np.abs(exact).max()
        assert err < bound, err
    with pytest.raises(sxl.SxlError):
        sxl.mixed_gemm_noalloc(640, "fp16", torch.zeros(2, 640, 640, dtype=torch.float64,
                                                        device="cuda"),
                               torch.zeros(2, 640, 640, dtype=torch.float64, device="cuda"))
    ctx.close()
