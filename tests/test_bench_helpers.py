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

