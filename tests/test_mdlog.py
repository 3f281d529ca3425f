"""The JSON-lines MD log (host logic; a stand-in context supplies the
library's per-step statistics, charges and step counter)."""
import json

import numpy as np
import pytest

from paper_2303_03529_gb300 import mdlog


def test_spin_moments_per_atom_and_per_shell():
    # 2 atoms, per atom: up = [5, 4], down = [3, 4] -> m = [2, 0]
    q = np.array([5.0, 4.0, 3.0, 4.0])
    np.testing.assert_array_equal(mdlog.spin_moments(q, 2), [2.0, 0.0])
    # shell-resolved: atom 0 shells up (1, 0, 4) down (1, 0, 2) -> m = 2;
    # atom 1 up (0.5, 0, 3) down (0.5, 0, 4) -> m = -1
    q = np.array([1, 0, 4, 0.5, 0, 3, 1, 0, 2, 0.5, 0, 4], dtype=float)
    np.testing.assert_allclose(mdlog.spin_moments(q, 2), [2.0, -1.0])
    with pytest.raises(ValueError):
        mdlog.spin_moments(np.zeros(10), 3)


def test_step_record_fields():
    rec = mdlog.step_record(7, [-80.0, 300.0, 1e-5, -4.9], 16, np.array([1.0, 0.0, 0.0, 0.5] * 8),
                            0.25)
    assert rec["step"] == 7 and rec["E_tot_per_atom"] == -5.0 and rec["T"] == 300.0
    assert rec["rms_q_minus_n"] == 1e-5 and rec["mu"] == -4.9
    assert rec["wall_s_per_step"] == 0.25
    assert set(rec) >= {"m_total", "m_abs_max"}


class _FakeContext:
    """Duck-typed library context: energies fall by 1 eV per step."""

    nat = 2

    def __init__(self):
        self.k = 0

    def step(self, n, stats=True):
        rows = []
        for _ in range(n):
            self.k += 1
            rows.append([-10.0 - self.k, 300.0 + self.k, 1e-4, -5.0])
        return np.array(rows)

    def charges(self):
        return np.array([0.6, 0.1, -0.6, -0.1])

    def md_step(self):
        return self.k


def test_run_writes_one_line_per_block(tmp_path):
    path = tmp_path / "md.jsonl"
    recs = mdlog.run(_FakeContext(), 5, path, every=2)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines == recs
    assert [r["step"] for r in lines] == [2, 4, 5]
    assert lines[-1]["E_tot_per_atom"] == -15.0 / 2
    assert lines[0]["m_total"] == pytest.approx(1.4)
    with pytest.raises(ValueError):
        mdlog.run(_FakeContext(), 3, path, every=0)


def test_spin_flip_events():
    def rec(step, rms, mt, ma):
        return {"step": step, "rms_q_minus_n": rms, "m_total": mt, "m_abs_max": ma}
    quiet = [rec(i, 1e-4, 32.0, 2.1) for i in range(5)]
    assert mdlog.spin_flip_events(quiet) == []
    flip = quiet + [rec(5, 3e-3, 30.0, 2.1), rec(6, 2e-4, 30.0, 2.1)]
    ev = mdlog.spin_flip_events(flip)
    assert (5, "residual jump") in ev and (5, "m_total jump") in ev
    assert all(s == 5 for s, _ in ev)
