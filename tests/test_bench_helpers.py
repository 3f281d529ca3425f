"""Host-side helpers of bench.py: the kernel-source hash that keys the
recorded ncu traffic ignores comments and whitespace but not code (a code
change makes bench.py report the traffic as null until it is re-measured)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_source_hash_ignores_comments_not_code(tmp_path):
    b = _bench()
    base = "int f(int x) {\n  return x + 1;  // one\n}\n/* block\n comment */\n"
    p1, p2, p3 = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    p1.write_text(base)
    p2.write_text(base.replace("// one", "// a different remark").replace("  return", "\treturn"))
    p3.write_text(base.replace("x + 1", "x + 2"))
    assert b.kernel_source_hash(str(p1)) == b.kernel_source_hash(str(p2))
    assert b.kernel_source_hash(str(p1)) != b.kernel_source_hash(str(p3))



def test_scaled_traffic_fits_two_captures():
    """Reads a n^3 + b n^2 through the two captured sizes, writes ~ n^2."""
    b = _bench()
    a3, b2, w2 = 3.0e-3, 40.0, 12.0
    n1, n2 = 2304, 4608
    rec = {"variants": {"plain": {"n": [n1, n2],
                                  "read_bytes": [a3 * n1 ** 3 + b2 * n1 ** 2,
                                                 a3 * n2 ** 3 + b2 * n2 ** 2],
                                  "write_bytes": [w2 * n1 ** 2, w2 * n2 ** 2]}}}
    for n in (n1, n2, 9216):
        expect = a3 * n ** 3 + b2 * n ** 2 + w2 * n ** 2
        assert abs(b.scaled_traffic(rec, "plain", n) - expect) < 1e-6 * expect
    assert b.scaled_traffic(rec, "dual", 9216) is None
    assert b.scaled_traffic(None, "plain", 9216) is None


def test_roofline_counts_each_product_once():
    """A split launch issues three MMAs per k step but is one product: the
    achieved rate and the fraction count product flops, not issued ones."""
    b = _bench()
    ms = 10.0
    flops = 2.0 * 2 * 1000 ** 3          # one product, both spins
    tm = {"tc_launches": 2, "tc_ms": 2 * ms, "tc_fp32_flops": 2 * flops,
          "tc_mma_flops": 4 * flops, "tc_alg_flops": 4 * flops}
    gt = {"plain": {"launches": 1, "ms": ms, "issued_flops": flops, "product_flops": flops},
          "dual": {"launches": 0, "ms": 0.0, "issued_flops": 0.0, "product_flops": 0.0},
          "split": {"launches": 1, "ms": ms, "issued_flops": 3 * flops, "product_flops": flops},
          "fp64": {"launches": 0, "ms": 0.0, "issued_flops": 0.0, "product_flops": 0.0}}
    r = b.roofline(tm, gt, 40.0, {"bf16_tflops_sustained": 1000.0}, "measured", None, None, "fp16")
    rate = flops / (ms / 1e3) / 1e12
    assert abs(r["achieved"] - rate) < 1e-6 and abs(r["frac"] - rate / 1000.0) < 1e-6
    assert abs(r["mma_issued_tflops"] - 2 * rate) < 1e-6
    assert r["per_form"]["split"]["issued_tflops"] == round(3 * rate, 1)
    assert r["per_form"]["split"]["achieved"] == round(rate, 1)
    assert r["share_of_step"] == 0.5 and r["traffic"] is None


def test_oracle_step_cycle_covers_every_component():
    """The reference arm's K timed steps each run one component of an oracle
    MD step; after complete() every component has a time and the step time
    is their sum (16-atom cell, a second of CPU)."""
    b = _bench()
    from paper_2303_03529_gb300 import workload
    st = b.OracleStep(workload.fe16())
    m = st.p.krylov_rank
    assert st.cycle == ["hamiltonian", "density", "forces", "energy"] + ["krylov"] * m + ["lsq"]
    for _ in range(3):
        st.next()
    extra = st.complete()
    assert extra == len(st.cycle) - 3
    assert all(t is not None and t >= 0 for t in st.times)
    assert abs(st.step_seconds() - sum(st.times)) < 1e-12
    assert st.kb is not None and len(st.kb.V) == m
