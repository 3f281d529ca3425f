"""The JSON configurations of the workloads (host logic, no GPU): every
committed file matches the code's workload, and regenerates its inputs bit
for bit."""
import dataclasses
import json
import os

import numpy as np
import pytest

from paper_2303_03529_gb300 import workload as wl

CONFIGS = os.path.join(os.path.dirname(wl.__file__), "configs")


@pytest.mark.parametrize("key", sorted(wl.WORKLOADS))
def test_committed_config_regenerates_the_workload(key):
    w = wl.WORKLOADS[key]()
    with open(os.path.join(CONFIGS, f"{key}.json")) as f:
        cfg = json.load(f)
    assert cfg == json.loads(json.dumps(wl.config(w)))  # no drift between file and code
    v = wl.from_config(cfg)
    for name in ("R", "V", "n0", "cell"):
        np.testing.assert_array_equal(getattr(v, name), getattr(w, name))
    assert v.params == w.params and v.name == w.name and v.steps == w.steps
    assert v.shell_resolved_n0 == w.shell_resolved_n0


def test_config_round_trip_and_rejections(tmp_path):
    w = wl.make_cell(3, seed=7, sigma=0.04, vacancy_frac=0.05, name="x",
                     params=wl.ModelParams(krylov_rank=5, kT=0.12))
    cfg = wl.config(w, precision="bf16")
    assert cfg["precision"] == "bf16" and cfg["params"]["krylov_rank"] == 5
    p = tmp_path / "x.json"
    p.write_text(json.dumps(cfg))
    v = wl.load_config(p)
    np.testing.assert_array_equal(v.R, w.R)
    assert v.n_atoms == w.n_atoms == 52 and v.params.kT == 0.12  # 54 sites, int(0.05 * 54) = 2 vacancies
    with pytest.raises(ValueError, match="unknown parameters"):
        wl.from_config(dict(cfg, params=dict(cfg["params"], bogus=1)))
    with pytest.raises(ValueError, match="unsupported"):
        wl.from_config(dict(cfg, version=99))
    # every field of the parameter set is in the file
    assert set(cfg["params"]) == {f.name for f in dataclasses.fields(wl.ModelParams)}
